// a2: tile/depth binning with a hand-written stable LSD radix sort.
//
// Eq. 1 blends "depth-sorted" Gaussians; with 16x16 tiles each tile needs the Gaussians
// covering it in (depth, id) order.  Instead of sorting all I (tile, depth) instances by
// a 64-bit key, the path sorts the N Gaussians once by depth (32-bit keys: culled ones
// carry 0xFFFFFFFF and sort last), emits the tile instances in that order, and
// stable-sorts the I instances by tile id only (ceil(log2 T) bits, one or two passes).
// Stability makes the result identical to a stable sort by (tile, depth) of instances
// emitted in id order.
//
// Each radix pass is a single kernel ("onesweep"): a block takes the next 4096-element
// chunk from a ticket counter, ranks its keys with warp match, publishes per-digit
// counts, and finds its per-digit output offset by decoupled look-back over the chunks
// before it (each poll is bounded; a wait that runs out sets an error bit and the block
// carries on with guarded writes).  Digit histograms of all passes are computed up front
// (depth keys) or while emitting the instances (tile keys).  The tile-count prefix sum
// is fused into the emission kernel with the same look-back.
#include "gs_blend.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kItemsBig = 16;               // elements per thread for large sorts
constexpr int kItemsSmall = 8;              // ... and below kSmallSort elements
constexpr int64_t kSmallSort = 1 << 21;
constexpr int kEmitItems = 8;
constexpr int kEmitChunk = kThreads * kEmitItems;   // 1024 Gaussians per emission block
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u, kFlagPre = 2u;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ int64_t dev_count(const uint32_t* d_n, int64_t bound) {
  return d_n ? min64((int64_t)*d_n, bound) : bound;
}

// Block-wide exclusive scan of one value per thread; returns the prefix, *total the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;   // inclusive warp prefixes
  }
  __syncthreads();
  const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0;
  *total = s_warp[kWarps - 1];
  __syncthreads();
  return before + x - v;
}

// Next chunk index from a ticket counter.  Chunks are handed out in launch order, so the
// chunks before any running block have all started.  The last taker resets the counter
// for the next launch (every other block has taken its ticket by then).
__device__ __forceinline__ int acquire_chunk(uint32_t* ticket, int nblocks, uint32_t* s_chunk) {
  if (threadIdx.x == 0) {
    const uint32_t c = atomicAdd(ticket, 1u);
    if (c == (uint32_t)nblocks - 1) atomicExch(ticket, 0u);
    *s_chunk = c;
  }
  __syncthreads();
  return (int)*s_chunk;
}

// Status word of the look-back: high 32 bits = epoch << 2 | flag, low 32 bits = value.
// Words of older launches (other epochs) read as "not yet published".
__device__ __forceinline__ void publish(unsigned long long* p, uint32_t epoch, uint32_t flag,
                                        uint32_t v) {
  atomicExch(p, ((unsigned long long)((epoch << 2) | flag) << 32) | v);
}

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ bool status_ready(unsigned long long w, uint32_t epoch) {
  const uint32_t hi = (uint32_t)(w >> 32);
  return (hi >> 2) == epoch && (hi & 3u) != 0u;
}

// Sum of the published values of the chunks before `chunk` in column `col`, walking back
// until an inclusive prefix is found.  The words of up to kLB predecessors are requested
// together, so a walk over many chunks costs a few memory round trips.  Each wait for a
// word not yet published is bounded.
constexpr int kLB = 8;
__device__ uint32_t look_back(const unsigned long long* status, int chunk, int col, int stride,
                              uint32_t epoch, uint32_t* err) {
  uint32_t excl = 0;
  for (int k = chunk - 1; k >= 0; k -= kLB) {
    unsigned long long w[kLB];
#pragma unroll
    for (int j = 0; j < kLB; ++j)
      w[j] = k - j >= 0 ? ld_status(status + (size_t)(k - j) * stride + col) : 0ull;
#pragma unroll
    for (int j = 0; j < kLB; ++j) {
      if (k - j < 0) break;
      int spins = 0;
      while (!status_ready(w[j], epoch)) {
        if (++spins > kSpinLimit) {
          atomicOr(err, kErrLookback);
          return excl;
        }
        if (spins > 32) __nanosleep(100);
        w[j] = ld_status(status + (size_t)(k - j) * stride + col);
      }
      excl += (uint32_t)w[j];
      if ((uint32_t)(w[j] >> 32 & 3u) == kFlagPre) return excl;
    }
  }
  return excl;
}

// ---------------------------------------------------------------- radix sort

// Digit histograms of all four 8-bit digits of the depth keys (grid-stride).
__global__ void __launch_bounds__(kThreads)
k_hist4(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t s_h[4 * kRadix];
  for (int e = threadIdx.x; e < 4 * kRadix; e += kThreads) s_h[e] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const uint32_t k = keys[i];
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p * kRadix + ((k >> (8 * p)) & 0xFFu)], 1u);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 4 * kRadix; e += kThreads)
    if (s_h[e]) atomicAdd(&ghist[e], s_h[e]);
}

// One stable LSD pass over 8 bits at `shift`.  Warp w owns elements [w*512, w*512+512) of
// the chunk in rounds of 32; lanes with equal digits are ranked with __match_any_sync.
// vin == nullptr means the values are the element indices.
template <int kItems>
__global__ void __launch_bounds__(kThreads)
k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* d_n,
           int64_t bound, int nblocks, int shift, const uint32_t* __restrict__ ghist,
           unsigned long long* __restrict__ status, uint32_t* ticket, uint32_t epoch,
           uint32_t* err) {
  __shared__ uint32_t s_wcnt[kWarps][kRadix];     // per-warp digit counts -> offsets
  __shared__ uint32_t s_dstart[kRadix];           // digit start inside the chunk
  __shared__ uint32_t s_gbase[kRadix];            // digit start in the output
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_chunk;
  constexpr int kChunk = kThreads * kItems;
  __shared__ uint32_t s_keys[kChunk];
  __shared__ uint32_t s_vals[kChunk];
  const int chunk = acquire_chunk(ticket, nblocks, &s_chunk);
  const int64_t n = dev_count(d_n, bound);
  const int64_t base = (int64_t)chunk * kChunk;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s_wcnt[0][0])[d] = 0;
  __syncthreads();

  uint32_t key[kItems], val[kItems], rank[kItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
  // all loads first (in flight together), then the ranking rounds
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + warp * (kItems * 32) + r * 32 + lane;
    key[r] = i < n ? kin[i] : 0u;
    val[r] = i < n ? (vin ? vin[i] : (uint32_t)i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + warp * (kItems * 32) + r * 32 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? ((key[r] >> shift) & 0xFFu) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? s_wcnt[warp][d] : 0u;
    rank[r] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wcnt[w][d];
      s_wcnt[w][d] = cnt;
      cnt += c;
    }
    unsigned long long* st = status + (size_t)chunk * kRadix + d;
    publish(st, epoch, chunk == 0 ? kFlagPre : kFlagAgg, cnt);
    uint32_t tot;
    const uint32_t dstart = block_exclusive_scan(cnt, s_warp, &tot);
    const uint32_t gpre = block_exclusive_scan(ghist[d], s_warp, &tot);
    uint32_t excl = 0;
    if (chunk > 0) {
      excl = look_back(status, chunk, d, kRadix, epoch, err);
      publish(st, epoch, kFlagPre, excl + cnt);
    }
    s_dstart[d] = dstart;
    s_gbase[d] = gpre + excl;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + warp * (kItems * 32) + r * 32 + lane;
    if (i < n) {
      const uint32_t d = (key[r] >> shift) & 0xFFu;
      const uint32_t pos = s_dstart[d] + s_wcnt[warp][d] + rank[r];
      s_keys[pos] = key[r];
      s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  const int cnt = (int)min64(kChunk, n - base);
  for (int j = threadIdx.x; j < cnt; j += kThreads) {
    const uint32_t k = s_keys[j];
    const uint32_t d = (k >> shift) & 0xFFu;
    const int64_t o = (int64_t)s_gbase[d] + j - s_dstart[d];
    if (o < n) {               // always true unless a look-back timed out
      kout[o] = k;
      vout[o] = s_vals[j];
    }
  }
}

// ---------------------------------------------------------------- instance emission

// Exclusive prefix of the tile counts of the depth-sorted Gaussians (decoupled look-back
// over chunks of kEmitChunk): offsets[r] = first instance slot of sorted Gaussian r.
__global__ void __launch_bounds__(kThreads)
k_tile_offsets(const uint32_t* __restrict__ sorted_ids, const uint32_t* __restrict__ ntiles,
               int64_t n, int nblocks, uint32_t* __restrict__ offsets,
               unsigned long long* __restrict__ status, uint32_t* ticket, uint32_t epoch,
               uint32_t* counters) {
  constexpr int EI = kEmitItems;
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_chunk, s_base;
  const int chunk = acquire_chunk(ticket, nblocks, &s_chunk);
  const int64_t i0 = (int64_t)chunk * kEmitChunk + threadIdx.x * EI;
  if ((int64_t)chunk * kEmitChunk >= n) return;
  uint32_t cnt[EI];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < EI; ++k) {
    const uint32_t id = i0 + k < n ? sorted_ids[i0 + k] : 0xFFFFFFFFu;
    cnt[k] = id < (uint32_t)n ? ntiles[id] : 0u;
    sum += cnt[k];
  }
  uint32_t total;
  uint32_t off = block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) {
    unsigned long long* st = status + chunk;
    publish(st, epoch, chunk == 0 ? kFlagPre : kFlagAgg, total);
    uint32_t excl = 0;
    if (chunk > 0) {
      excl = look_back(status, chunk, 0, 1, epoch, &counters[kCntStatus]);
      publish(st, epoch, kFlagPre, excl + total);
    }
    s_base = excl;
  }
  __syncthreads();
  off += s_base;
#pragma unroll
  for (int k = 0; k < EI; ++k) {
    if (i0 + k < n) offsets[i0 + k] = off;
    off += cnt[k];
  }
}

// Instance emission balanced over output slots: thread t of block b writes slots
// [b*kEmitChunk + t*kEmitItems, + kEmitItems).  The Gaussian owning a slot is the last r
// with offsets[r] <= slot (binary search for the first slot, then a forward walk).  Each
// Gaussian's slots hold its tiles in row-major order.  Also accumulates the three 8-bit
// digit histograms of the tile ids for the tile sort.  Slots at or beyond min(I, cap)
// are not written; I above cap is flagged.
__global__ void __launch_bounds__(kThreads)
k_emit(const uint32_t* __restrict__ sorted_ids, const uint32_t* __restrict__ offsets,
       const uint2* __restrict__ rect, int64_t n, int TX, int64_t cap,
       uint32_t* __restrict__ inst_tile, uint32_t* __restrict__ inst_id,
       uint32_t* __restrict__ ghist_tile, uint32_t* counters) {
  __shared__ uint32_t s_h[3 * kRadix];
  for (int e = threadIdx.x; e < 3 * kRadix; e += kThreads) s_h[e] = 0;
  __syncthreads();
  const int64_t I = (int64_t)counters[kCntInst];
  if (threadIdx.x == 0 && blockIdx.x == 0 && I > cap) atomicOr(&counters[kCntStatus], kErrInstOverflow);
  const int64_t m = min64(I, cap);
  const int64_t o0 = (int64_t)blockIdx.x * kEmitChunk + threadIdx.x * kEmitItems;
  if (o0 < m && n > 0) {
    // last r with offsets[r] <= o0
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= (uint32_t)o0) lo = mid; else hi = mid - 1;
    }
    int64_t r = lo;
    uint32_t id = sorted_ids[r];
    uint2 rc = id < (uint32_t)n ? rect[id] : make_uint2(0u, 0u);
    uint32_t start = offsets[r];
#pragma unroll 1
    for (int k = 0; k < kEmitItems; ++k) {
      const int64_t o = o0 + k;
      if (o >= m) break;
      while (r + 1 < n && offsets[r + 1] <= (uint32_t)o) {
        ++r;
        id = sorted_ids[r];
        rc = id < (uint32_t)n ? rect[id] : make_uint2(0u, 0u);
        start = offsets[r];
      }
      const uint32_t x0 = rc.x & 0xFFFFu, y0 = rc.x >> 16, w = (rc.y & 0xFFFFu) - x0;
      if (w == 0u) continue;    // inconsistent inputs only
      const uint32_t q = (uint32_t)o - start;
      const uint32_t t = (y0 + q / w) * (uint32_t)TX + x0 + q % w;
      inst_tile[o] = t;
      inst_id[o] = id;
      atomicAdd(&s_h[t & 0xFFu], 1u);
      atomicAdd(&s_h[kRadix + ((t >> 8) & 0xFFu)], 1u);
      atomicAdd(&s_h[2 * kRadix + ((t >> 16) & 0xFFu)], 1u);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * kRadix; e += kThreads)
    if (s_h[e]) atomicAdd(&ghist_tile[e], s_h[e]);
}

__global__ void k_ranges(const uint32_t* __restrict__ tile, const uint32_t* counters, int64_t bound,
                         int64_t cap, int n_tiles, uint2* __restrict__ ranges) {
  const int64_t n = min64(min64((int64_t)counters[kCntInst], bound), cap);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = tile[i];
  if (t >= (uint32_t)n_tiles) {
    atomicOr((uint32_t*)&counters[kCntStatus], kErrBadRange);
    return;
  }
  if (i == 0 || tile[i - 1] != t) ranges[t].x = (uint32_t)i;
  if (i + 1 == n || tile[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

// Heavy-first tile order for the persistent raster kernels: tiles bucketed by the bit
// length of their list length, longest buckets first (order inside a bucket is arbitrary;
// results do not depend on the order tiles are processed in).  One block.
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads)
k_tile_order(const uint2* __restrict__ ranges, int n_tiles, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_cnt[33], s_cur[33];
  if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    atomicAdd(&s_cnt[__clz((int)(r.y - r.x))], 1u);   // 32 - bit length: longest first
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int b = 0; b < 33; ++b) {
      s_cur[b] = acc;
      acc += s_cnt[b];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    order[atomicAdd(&s_cur[__clz((int)(r.y - r.x))], 1u)] = (uint32_t)t;
  }
}

// Statistics for the roofline model (not on the rendering path): per pixel, the list
// entries up to its last contributor (the pairs the backward pass evaluates) and how many
// of them it blended, summed over the image into stats64[0..1].  The opacity test is the
// rasterizer's own (gs_blend.cuh).
__global__ void __launch_bounds__(kThreads)
k_pair_stats(CamDev cam, const GaussRec* __restrict__ rec, const uint2* __restrict__ ranges,
             const uint32_t* __restrict__ inst_id, const uint32_t* __restrict__ n_contrib,
             unsigned long long* __restrict__ stats64) {
  const int tile = blockIdx.x;
  const int px = (tile % cam.TX) * 16 + (threadIdx.x & 15), py = (tile / cam.TX) * 16 + (threadIdx.x >> 4);
  uint32_t eval = 0, blend = 0;
  if (px < cam.W && py < cam.H) {
    const uint32_t nc = n_contrib[(int64_t)py * cam.W + px];
    const uint2 rg = ranges[tile];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    for (uint32_t k = 0; k < nc && rg.x + k < rg.y; ++k) {
      const uint32_t id = inst_id[rg.x + k];
      if (id >= (uint32_t)cam.n_gauss) continue;
      const float4 r0 = rec[id].r0, r1 = rec[id].r1;
      ++eval;
      const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
      if (sigma >= 0.f && fminf(kAlphaMax, __fmul_rn(r1.y, blend_gauss(sigma))) >= kAlphaMin) ++blend;
    }
  }
  __shared__ unsigned long long s[2];
  if (threadIdx.x == 0) s[0] = s[1] = 0ull;
  __syncthreads();
  eval = __reduce_add_sync(0xffffffffu, eval);
  blend = __reduce_add_sync(0xffffffffu, blend);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s[0], (unsigned long long)eval);
    atomicAdd(&s[1], (unsigned long long)blend);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&stats64[0], s[0]);
    atomicAdd(&stats64[1], s[1]);
  }
}

// I_eff = sum over tiles of max n_contrib inside the tile.
__global__ void __launch_bounds__(kThreads)
k_inst_eff(const uint32_t* __restrict__ n_contrib, int TX, int W, int H, uint32_t* counters) {
  const int tile = blockIdx.x;
  const int px = (tile % TX) * 16 + (threadIdx.x & 15), py = (tile / TX) * 16 + (threadIdx.x >> 4);
  uint32_t v = (px < W && py < H) ? n_contrib[(int64_t)py * W + px] : 0u;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ uint32_t s[kWarps];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0;
    for (int w = 0; w < kWarps; ++w) m = max(m, s[w]);
    atomicAdd(&counters[kCntInstEff], m);
  }
}

int sort_items(int64_t n) { return n >= kSmallSort ? kItemsBig : kItemsSmall; }
int num_chunks(int64_t n, int items) { return (int)ceil_div(max64(n, 1), (int64_t)kThreads * items); }

// One onesweep pass with the chunk size chosen for n.
void onesweep(int items, int nb, cudaStream_t st, const uint32_t* kin, const uint32_t* vin,
              uint32_t* kout, uint32_t* vout, const uint32_t* d_n, int64_t bound, int shift,
              const uint32_t* ghist, const BinScratch& s, uint32_t* ticket) {
  if (items == kItemsBig)
    k_onesweep<kItemsBig><<<nb, kThreads, 0, st>>>(kin, vin, kout, vout, d_n, bound, nb, shift, ghist,
                                                   s.status, ticket, s.next_epoch(),
                                                   s.counters + kCntStatus);
  else
    k_onesweep<kItemsSmall><<<nb, kThreads, 0, st>>>(kin, vin, kout, vout, d_n, bound, nb, shift, ghist,
                                                     s.status, ticket, s.next_epoch(),
                                                     s.counters + kCntStatus);
  note_launch();
}

}  // namespace

// Enough for any n <= max_elems: the smallest chunk (kItemsSmall == kEmitItems) gives the
// most chunks, each needing kRadix words.
size_t bin_status_words(int64_t max_elems) {
  static_assert(kEmitItems == kItemsSmall, "status sizing assumes the smallest chunk");
  return (size_t)num_chunks(max_elems, kItemsSmall) * kRadix;
}

void launch_depth_sort(const uint32_t* depth_key, int64_t n, uint32_t* k1, uint32_t* v1,
                       uint32_t* k0, uint32_t* v0, const BinScratch& s, cudaStream_t st) {
  if (n <= 0) return;
  const int items = sort_items(n);
  const int nb = num_chunks(n, items);
  k_hist4<<<std::min(nb, 4 * 152), kThreads, 0, st>>>(depth_key, n, s.ghist);
  note_launch();
  // pass 0 reads the projection's keys and generates the ids; passes alternate 1 <-> 0
  const uint32_t* ki = depth_key;
  const uint32_t* vi = nullptr;
  uint32_t* ko[4] = {k1, k0, k1, k0};
  uint32_t* vo[4] = {v1, v0, v1, v0};
  for (int p = 0; p < 4; ++p) {
    onesweep(items, nb, st, ki, vi, ko[p], vo[p], nullptr, n, 8 * p, s.ghist + p * kRadix, s,
             s.tickets);
    ki = ko[p];
    vi = vo[p];
  }
}

void launch_emit_instances(const uint32_t* sorted_ids, const uint32_t* ntiles, const uint2* rect,
                           int64_t n, int TX, int64_t cap, uint32_t* offsets, uint32_t* inst_tile,
                           uint32_t* inst_id, const BinScratch& s, cudaStream_t st) {
  if (n <= 0) return;
  const int nb = num_chunks(n, kEmitItems);
  k_tile_offsets<<<nb, kThreads, 0, st>>>(sorted_ids, ntiles, n, nb, offsets, s.status,
                                          s.tickets + 1, s.next_epoch(), s.counters);
  const int64_t slots = cap > 0 ? cap : 1;
  k_emit<<<num_chunks(slots, kEmitItems), kThreads, 0, st>>>(sorted_ids, offsets, rect, n, TX, cap,
                                                             inst_tile, inst_id, s.ghist + 4 * kRadix,
                                                             s.counters);
  note_launch(2);
}

int launch_tile_sort(int64_t bound, int tile_bits, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                     uint32_t* v1, const BinScratch& s, cudaStream_t st) {
  if (bound <= 0 || tile_bits <= 0) return 0;
  const int items = sort_items(bound);
  const int nb = num_chunks(bound, items);
  int cur = 0;
  for (int p = 0; p * 8 < tile_bits && p < 3; ++p) {
    onesweep(items, nb, st, cur ? k1 : k0, cur ? v1 : v0, cur ? k0 : k1, cur ? v0 : v1,
             s.counters + kCntInst, bound, 8 * p, s.ghist + (4 + p) * kRadix, s, s.tickets + 2);
    cur ^= 1;
  }
  return cur;
}

void launch_tile_ranges(const uint32_t* inst_tile, const uint32_t* counters, int64_t bound_i,
                        int64_t cap, int n_tiles, uint2* ranges, cudaStream_t st) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, st);
  const int64_t b = min64(bound_i, cap);
  if (b <= 0) return;
  k_ranges<<<(int)ceil_div(b, 256), 256, 0, st>>>(inst_tile, counters, bound_i, cap, n_tiles,
                                                   ranges);
  note_launch();
}

void launch_pair_stats(const CamDev& cam, const GaussRec* rec, const uint2* ranges,
                       const uint32_t* inst_id, const uint32_t* n_contrib,
                       unsigned long long* stats64, cudaStream_t st) {
  cudaMemsetAsync(stats64, 0, 2 * sizeof(unsigned long long), st);
  if (cam.TX * cam.TY == 0) return;
  k_pair_stats<<<cam.TX * cam.TY, kThreads, 0, st>>>(cam, rec, ranges, inst_id, n_contrib, stats64);
  note_launch();
}

bool launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, cudaStream_t st) {
  if (n_tiles <= 0 || n_tiles > kMaxOrderedTiles) return false;
  k_tile_order<<<1, kOrderThreads, 0, st>>>(ranges, n_tiles, order);
  note_launch();
  return true;
}

void launch_inst_eff(const uint32_t* n_contrib, int TX, int TY, int W, int H, uint32_t* counters,
                     cudaStream_t st) {
  cudaMemsetAsync(counters + kCntInstEff, 0, 4, st);
  if (TX * TY > 0) {
    k_inst_eff<<<TX * TY, kThreads, 0, st>>>(n_contrib, TX, W, H, counters);
    note_launch();
  }
}

}  // namespace gs
