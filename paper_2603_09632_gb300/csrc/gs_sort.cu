// a2: tile/depth binning with a hand-written stable LSD radix sort.
//
// Eq. 1 blends "depth-sorted" Gaussians; with 16x16 tiles each tile needs the Gaussians
// covering it in (depth, id) order.  Instead of sorting all I (tile, depth) instances by
// a 64-bit key, the path sorts the V visible Gaussians once by depth (32-bit keys, four
// 8-bit passes), emits their tile instances in that order, and stable-sorts the I
// instances by tile id only (ceil(log2 T) bits, one or two passes).  Stability makes the
// result identical to a stable sort by (tile, depth) of instances emitted in id order.
//
// Radix pass = reduce-then-scan: (1) per 4096-element chunk digit histograms, (2) one
// device-wide exclusive scan over the digit-major histogram, (3) a stable scatter that
// ranks elements with warp match/ballot, sorts the chunk locally in shared memory and
// writes each digit's run contiguously.  No kernel waits on another block.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kChunk = kThreads * kItems;   // 4096 elements per block
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;

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

// ---------------------------------------------------------------- device-wide scan
// Each block owns kChunk consecutive elements.

// The kItems consecutive elements [i0, i0 + kItems) of a thread, zero past n; 16-byte
// loads when the whole run is in range (buffers are 16-byte aligned, i0 is a multiple of 16).
__device__ __forceinline__ void load_run(const uint32_t* in, int64_t i0, int64_t n, uint32_t* v) {
  if (i0 + kItems <= n) {
    const uint4* p = reinterpret_cast<const uint4*>(in + i0);
#pragma unroll
    for (int k = 0; k < kItems / 4; ++k) {
      const uint4 q = p[k];
      v[4 * k] = q.x;
      v[4 * k + 1] = q.y;
      v[4 * k + 2] = q.z;
      v[4 * k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kItems; ++k) v[k] = i0 + k < n ? in[i0 + k] : 0u;
  }
}

__global__ void __launch_bounds__(kThreads)
k_scan_reduce(const uint32_t* __restrict__ in, const uint32_t* d_n, int64_t bound,
              uint32_t* __restrict__ partial) {
  __shared__ uint32_t s_warp[kWarps];
  const int64_t n = dev_count(d_n, bound);
  const int64_t i0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kItems;
  uint32_t v[kItems];
  load_run(in, i0, n, v);
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) sum += v[k];
  uint32_t total;
  block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Single block: exclusive scan of nblocks partial sums in place; grand total to *total_out.
__global__ void __launch_bounds__(kThreads)
k_scan_partials(uint32_t* __restrict__ partial, int nblocks, uint32_t* total_out) {
  __shared__ uint32_t s_warp[kWarps];
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nblocks; b0 += kThreads) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < nblocks ? partial[i] : 0;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, s_warp, &tot);
    if (i < nblocks) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(kThreads)
k_scan_down(const uint32_t* in, uint32_t* out, const uint32_t* d_n, int64_t bound,
            const uint32_t* __restrict__ partial) {
  __shared__ uint32_t s_warp[kWarps];
  const int64_t n = dev_count(d_n, bound);
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  if (base >= n) return;
  const int64_t i0 = base + (int64_t)threadIdx.x * kItems;
  uint32_t v[kItems];
  load_run(in, i0, n, v);
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) sum += v[k];
  uint32_t tot;
  uint32_t run = partial[blockIdx.x] + block_exclusive_scan(sum, s_warp, &tot);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const uint32_t x = v[k];
    v[k] = run;
    run += x;
  }
  if (i0 + kItems <= n) {
    uint4* q = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
    for (int k = 0; k < kItems / 4; ++k) q[k] = make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kItems; ++k)
      if (i0 + k < n) out[i0 + k] = v[k];
  }
}

void scan_impl(const uint32_t* in, uint32_t* out, const uint32_t* d_n, int64_t bound,
               uint32_t* temp, uint32_t* total_out, cudaStream_t st) {
  if (bound <= 0) {
    if (total_out) cudaMemsetAsync(total_out, 0, 4, st);
    return;
  }
  const int nb = (int)ceil_div(bound, kChunk);
  k_scan_reduce<<<nb, kThreads, 0, st>>>(in, d_n, bound, temp);
  k_scan_partials<<<1, kThreads, 0, st>>>(temp, nb, total_out);
  k_scan_down<<<nb, kThreads, 0, st>>>(in, out, d_n, bound, temp);
  note_launch(3);
}

// ---------------------------------------------------------------- radix sort passes

__global__ void __launch_bounds__(kThreads)
k_radix_hist(const uint32_t* __restrict__ keys, const uint32_t* d_n, int64_t bound, int shift,
             int nchunks, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_h[kRadix];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = dev_count(d_n, bound);
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nchunks + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one chunk.  Warp w owns elements [w*512, w*512+512) of the chunk, in
// rounds of 32; within a round lanes with equal digits are ranked with __match_any_sync.
__global__ void __launch_bounds__(kThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* d_n,
                int64_t bound, int shift, int nchunks, const uint32_t* __restrict__ hist_scan) {
  __shared__ uint32_t s_wcnt[kWarps][kRadix];     // per-warp digit counts -> offsets
  __shared__ uint32_t s_dstart[kRadix];           // digit start inside the chunk
  __shared__ uint32_t s_gbase[kRadix];            // digit start in the output
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_keys[kChunk];
  __shared__ uint32_t s_vals[kChunk];
  const int64_t n = dev_count(d_n, bound);
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s_wcnt[0][0])[d] = 0;
  __syncthreads();

  uint32_t key[kItems], val[kItems], rank[kItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + warp * (kItems * 32) + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? kin[i] : 0u;
    val[r] = valid ? vin[i] : 0u;
    const uint32_t d = valid ? ((key[r] >> shift) & 0xFFu) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? s_wcnt[warp][d] : 0u;
    rank[r] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive scan over warps, digit totals, chunk-local digit starts
  {
    const int d = threadIdx.x;
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wcnt[w][d];
      s_wcnt[w][d] = sum;
      sum += c;
    }
    uint32_t tot;
    const uint32_t start = block_exclusive_scan(sum, s_warp, &tot);
    s_dstart[d] = start;
    s_gbase[d] = hist_scan[(int64_t)d * nchunks + blockIdx.x];
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
    const uint32_t o = s_gbase[d] + (uint32_t)j - s_dstart[d];
    kout[o] = k;
    vout[o] = s_vals[j];
  }
}

// ---------------------------------------------------------------- binning kernels

__global__ void k_visible_flags(const uint32_t* __restrict__ ntiles, int64_t n,
                                uint32_t* __restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = ntiles[i] > 0 ? 1u : 0u;
}

__global__ void k_compact(const uint32_t* __restrict__ ntiles, const uint32_t* __restrict__ depth_key,
                          const uint32_t* __restrict__ pos, int64_t n, uint32_t* __restrict__ okeys,
                          uint32_t* __restrict__ oids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && ntiles[i] > 0) {
    const uint32_t p = pos[i];
    okeys[p] = depth_key[i];
    oids[p] = (uint32_t)i;
  }
}

__global__ void k_gather_counts(const uint32_t* __restrict__ sorted_ids,
                                const uint32_t* __restrict__ ntiles, const uint32_t* d_v,
                                int64_t bound, uint32_t* __restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < dev_count(d_v, bound)) cnt[r] = ntiles[sorted_ids[r]];
}

__global__ void k_emit(const uint32_t* __restrict__ sorted_ids, const uint2* __restrict__ rect,
                       const uint32_t* __restrict__ offsets, const uint32_t* d_v, int64_t bound,
                       int TX, uint32_t* counters, int64_t cap, uint32_t* __restrict__ inst_tile,
                       uint32_t* __restrict__ inst_id) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= dev_count(d_v, bound)) return;
  const uint32_t id = sorted_ids[r];
  const uint2 rc = rect[id];
  const int x0 = rc.x & 0xFFFF, y0 = rc.x >> 16, x1 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  int64_t o = offsets[r];
  bool overflow = false;
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx, ++o) {
      if (o < cap) {
        inst_tile[o] = (uint32_t)(ty * TX + tx);
        inst_id[o] = id;
      } else {
        overflow = true;
      }
    }
  if (overflow) atomicOr(&counters[kCntStatus], kErrInstOverflow);
}

__global__ void k_ranges(const uint32_t* __restrict__ tile, const uint32_t* counters, int64_t bound,
                         int64_t cap, uint2* __restrict__ ranges) {
  const int64_t n = min64(min64((int64_t)counters[kCntInst], bound), cap);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = tile[i];
  if (i == 0 || tile[i - 1] != t) ranges[t].x = (uint32_t)i;
  if (i + 1 == n || tile[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
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

}  // namespace

size_t scan_temp_words(int64_t n) { return (size_t)ceil_div(max64(n, 1), kChunk) + 32; }

void device_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* temp,
                           cudaStream_t st) {
  scan_impl(in, out, nullptr, n, temp, nullptr, st);
}

size_t radix_hist_words(int64_t bound) {
  return (size_t)kRadix * (size_t)ceil_div(max64(bound, 1), kChunk);
}

int radix_sort_pairs(const uint32_t* d_n, int64_t bound, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                     uint32_t* v1, int end_bit, uint32_t* hist, uint32_t* scan_temp,
                     cudaStream_t st) {
  if (bound <= 0 || end_bit <= 0) return 0;
  const int nchunks = (int)ceil_div(bound, kChunk);
  const int64_t hwords = (int64_t)kRadix * nchunks;
  int cur = 0;
  for (int shift = 0; shift < end_bit; shift += 8) {
    const uint32_t* ki = cur ? k1 : k0;
    const uint32_t* vi = cur ? v1 : v0;
    uint32_t* ko = cur ? k0 : k1;
    uint32_t* vo = cur ? v0 : v1;
    k_radix_hist<<<nchunks, kThreads, 0, st>>>(ki, d_n, bound, shift, nchunks, hist);
    scan_impl(hist, hist, nullptr, hwords, scan_temp, nullptr, st);
    k_radix_scatter<<<nchunks, kThreads, 0, st>>>(ki, vi, ko, vo, d_n, bound, shift, nchunks, hist);
    note_launch(2);
    cur ^= 1;
  }
  return cur;
}

void launch_compact_visible(const uint32_t* ntiles, const uint32_t* depth_key, int64_t n,
                            uint32_t* flags_scan, uint32_t* out_keys, uint32_t* out_ids,
                            uint32_t* counters, uint32_t* scan_temp, cudaStream_t st) {
  if (n <= 0) {
    cudaMemsetAsync(counters + kCntVisible, 0, 4, st);
    return;
  }
  const int g = (int)ceil_div(n, 256);
  k_visible_flags<<<g, 256, 0, st>>>(ntiles, n, flags_scan);
  scan_impl(flags_scan, flags_scan, nullptr, n, scan_temp, counters + kCntVisible, st);
  k_compact<<<g, 256, 0, st>>>(ntiles, depth_key, flags_scan, n, out_keys, out_ids);
  note_launch(2);
}

void launch_tile_offsets(const uint32_t* sorted_ids, const uint32_t* ntiles, int64_t bound_v,
                         uint32_t* counters, uint32_t* offsets, uint32_t* scan_temp,
                         cudaStream_t st) {
  if (bound_v <= 0) {
    cudaMemsetAsync(counters + kCntInst, 0, 4, st);
    return;
  }
  k_gather_counts<<<(int)ceil_div(bound_v, 256), 256, 0, st>>>(sorted_ids, ntiles,
                                                               counters + kCntVisible, bound_v,
                                                               offsets);
  note_launch();
  scan_impl(offsets, offsets, counters + kCntVisible, bound_v, scan_temp, counters + kCntInst, st);
}

void launch_emit_instances(const uint32_t* sorted_ids, const uint2* rect, const uint32_t* offsets,
                           int64_t bound_v, int TX, uint32_t* counters, int64_t cap,
                           uint32_t* inst_tile, uint32_t* inst_id, cudaStream_t st) {
  if (bound_v <= 0) return;
  k_emit<<<(int)ceil_div(bound_v, 256), 256, 0, st>>>(sorted_ids, rect, offsets,
                                                      counters + kCntVisible, bound_v, TX,
                                                      counters, cap, inst_tile, inst_id);
  note_launch();
}

void launch_tile_ranges(const uint32_t* inst_tile, const uint32_t* counters, int64_t bound_i,
                        int64_t cap, int n_tiles, uint2* ranges, cudaStream_t st) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, st);
  const int64_t b = min64(bound_i, cap);
  if (b <= 0) return;
  k_ranges<<<(int)ceil_div(b, 256), 256, 0, st>>>(inst_tile, counters, bound_i, cap, ranges);
  note_launch();
}

void launch_inst_eff(const uint2* ranges, const uint32_t* n_contrib, int TX, int TY, int W, int H,
                     uint32_t* counters, cudaStream_t st) {
  (void)ranges;
  cudaMemsetAsync(counters + kCntInstEff, 0, 4, st);
  if (TX * TY > 0) {
    k_inst_eff<<<TX * TY, kThreads, 0, st>>>(n_contrib, TX, W, H, counters);
    note_launch();
  }
}

}  // namespace gs
