// a2: tile/depth binning with a hand-written radix sort per tile.
//
// Eq. 1 blends "depth-sorted" Gaussians; with 16x16 tiles each tile needs the Gaussians
// covering it in (depth, id) order.  The frames of this path have a few thousand tiles
// holding tens to a few thousand instances each, so instead of global radix passes over
// all instances (each pass a chain of block-to-block dependencies) the binning works in
// tile buckets:
//   1. count: every visible Gaussian adds 1 to each tile of its rectangle (done by the
//      projection kernel, which has the rectangles in registers);
//   2. scan: one block turns the counts into tile ranges [start, end) and a heavy-first
//      tile order for the persistent raster kernels;
//   3. scatter: every (Gaussian, tile) instance takes a slot in its tile's range
//      (unordered) and stores the Gaussian's depth key and id there as one 8-byte pair;
//   4. sort: one block per tile sorts its range by depth with a stable LSD radix sort in
//      shared memory (8-bit digits; a pass whose digit is the same for the whole range is
//      skipped), then orders runs of equal depth by id, which makes the order the total
//      (depth, id) order whatever order the scatter left, and writes the sorted ids back.
//      Ranges longer than shared memory holds are sorted in chunks through global
//      ping-pong buffers.
// Steps 1 and 3 (warp_tile_instances) flatten the instances of a warp's 32 Gaussians and
// aggregate the atomic additions of equal tiles within a warp, so a Gaussian covering many
// tiles is spread over the warp instead of serialising one thread.
#include "gs_blend.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;
static_assert(kThreads == kRadix, "one thread per digit in the scans");
constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 16;                    // tiles per scan thread per round
constexpr int kSeg = 2048;                      // range size sorted in shared memory
constexpr int kSegRounds = kSeg / kThreads;     // elements per thread of a chunk

// Heavy-first order key of a tile with `count` instances: longest lists first, exact up to
// 1023 entries (longer lists share the first bucket).
__device__ __forceinline__ int order_key(uint32_t count) {
  return kScanThreads - 1 - (int)min(count, (uint32_t)(kScanThreads - 1));
}

// Row pass of the tile counts: the projection left per-row differences (TY rows of TX + 1
// words, +1 where a rectangle's row starts and -1 past its end); each row becomes its
// inclusive prefix sums in place, i.e. the tile counts at tile_slot(i), and the word past
// the row's last tile is cleared.  One warp per row.
__global__ void __launch_bounds__(kThreads)
k_bin_rows(uint32_t* __restrict__ tile_diff, int TX, int TY) {
  const int row = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= TY) return;   // uniform over the warp
  uint32_t* r = tile_diff + (int64_t)row * (TX + 1);
  uint32_t carry = 0;
  for (int x0 = 0; x0 < TX; x0 += 32) {
    const int x = x0 + lane;
    uint32_t v = x < TX ? r[x] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    if (x < TX) r[x] = carry + v;
    carry += __shfl_sync(kFull, v, 31);
  }
  if (lane == 0) r[TX] = 0u;
}

// Exclusive scan of the tile counts -> ranges (clamped to the instance capacity), write
// cursors, the overflow flag, and the heavy-first order (a counting sort of the tiles by
// list length, longest first; the order inside a bucket is arbitrary and results do not
// depend on it).  The counts are zeroed after their last read, ready for the next
// projection.  One block.
__global__ void __launch_bounds__(kScanThreads)
k_bin_scan(uint32_t* __restrict__ tile_count, int n_tiles, int TX, int64_t cap,
           uint2* __restrict__ ranges, uint32_t* __restrict__ cursor, uint32_t* __restrict__ order,
           uint32_t* counters) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_carry;
  __shared__ uint32_t s_b[kScanThreads];   // order buckets: tiles per list length
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_carry = 0;
  s_b[t] = 0;
  __syncthreads();
  for (int r0 = 0; r0 < n_tiles; r0 += kScanThreads * kScanPer) {
    const int i0 = r0 + t * kScanPer;
    uint32_t c[kScanPer];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      c[j] = i0 + j < n_tiles ? tile_count[tile_slot(i0 + j, TX)] : 0u;
      if (!order && i0 + j < n_tiles) tile_count[tile_slot(i0 + j, TX)] = 0u;   // last read without an order
      sum += c[j];
      if (order) {   // bucket histogram: one shared atomic per distinct bucket per warp
        const int key = i0 + j < n_tiles ? order_key(c[j]) : kScanThreads;
        const unsigned peers = __match_any_sync(kFull, key);
        if (key < kScanThreads && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&s_b[key], (uint32_t)__popc(peers));
      }
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;   // inclusive prefixes of the 32 warps
    }
    __syncthreads();
    uint32_t off = s_carry + (warp ? s_warp[warp - 1] : 0u) + x - sum;
    const uint32_t round_total = s_warp[kScanThreads / 32 - 1];
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      if (i0 + j < n_tiles) {
        const int64_t s = min64(off, cap), e = min64((int64_t)off + c[j], cap);
        // an empty tile reads as [0, 0)
        ranges[i0 + j] = c[j] ? make_uint2((uint32_t)s, (uint32_t)e) : make_uint2(0u, 0u);
        cursor[i0 + j] = off;
      }
      off += c[j];
    }
    __syncthreads();
    if (t == 0) s_carry += round_total;
    __syncthreads();
  }
  if (t == 0 && (int64_t)s_carry > cap) atomicOr(&counters[kCntStatus], kErrInstOverflow);
  if (!order) return;
  {   // exclusive scan of the order buckets, one per thread
    const uint32_t v = s_b[t];
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    s_b[t] = (warp ? s_warp[warp - 1] : 0u) + x - v;
  }
  __syncthreads();
  for (int i0 = 0; i0 < n_tiles; i0 += kScanThreads) {   // warp-aggregated bucket slots
    const int i = i0 + t;
    const int key = i < n_tiles ? order_key(tile_count[tile_slot(i, TX)]) : kScanThreads;
    if (i < n_tiles) tile_count[tile_slot(i, TX)] = 0u;   // last read
    const unsigned peers = __match_any_sync(kFull, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (key < kScanThreads && lane == leader) base = atomicAdd(&s_b[key], (uint32_t)__popc(peers));
    base = __shfl_sync(kFull, base, leader);
    if (i < n_tiles) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// Every instance takes a slot in its tile's range (one atomic per distinct tile per warp
// round) and stores the Gaussian's depth key and id.  The slot atomics of up to kScatterR
// rounds are issued before their stores, so their latencies overlap.  Slots at or beyond
// the capacity are not written.
constexpr int kScatterR = 4;
__global__ void __launch_bounds__(kThreads)
k_bin_scatter(int64_t n, const uint32_t* __restrict__ ntiles, const uint2* __restrict__ rect,
              const uint32_t* __restrict__ depth_key, int TX, int n_tiles, int64_t cap,
              uint32_t* __restrict__ cursor, uint2* __restrict__ inst_kv) {
  const int lane = threadIdx.x & 31;
  const int64_t g0 = (int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31);
  const int64_t gl = g0 + lane;
  const uint32_t nt = gl < n ? ntiles[gl] : 0u;
  const WarpInstances wi = warp_instances_begin(nt, nt ? rect[gl] : make_uint2(0u, 0u));
  for (uint32_t b0 = 0; b0 < wi.total; b0 += 32 * kScatterR) {
    uint32_t tile[kScatterR], peers[kScatterR], base[kScatterR];
    int owner[kScatterR];
#pragma unroll
    for (int r = 0; r < kScatterR; ++r) {
      tile[r] = 0xFFFFFFFFu;
      peers[r] = 0u;
      base[r] = 0u;
      owner[r] = 0;
      if (b0 + 32u * r < wi.total) {   // uniform over the warp
        tile[r] = warp_instance_tile(wi, b0 + 32u * r + lane, TX, &owner[r]);
        const bool ok = tile[r] < (uint32_t)n_tiles;
        peers[r] = __match_any_sync(kFull, ok ? tile[r] : 0xFFFFFFFFu);
        if (ok && lane == __ffs(peers[r]) - 1) base[r] = atomicAdd(&cursor[tile[r]], (uint32_t)__popc(peers[r]));
      }
    }
#pragma unroll
    for (int r = 0; r < kScatterR; ++r) {
      if (b0 + 32u * r < wi.total) {
        const uint32_t bs = __shfl_sync(kFull, base[r], __ffs(peers[r]) - 1);
        if (tile[r] < (uint32_t)n_tiles) {
          const uint32_t pos = bs + __popc(peers[r] & ((1u << lane) - 1u));
          if ((int64_t)pos < cap) {
            const int64_t g = g0 + owner[r];
            inst_kv[pos] = make_uint2(depth_key[g], (uint32_t)g);   // one 8-byte store
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- per-tile radix sort

// Stable destinations of one chunk of cnt <= kSeg keys by the 8-bit digit at `shift`.
// Warp w owns the contiguous elements [w * 32 R, (w + 1) * 32 R), R = ceil(cnt / 256),
// taken in rounds of 32; lanes with equal digits are ranked with __match_any_sync.  On
// return pos[r] is the chunk-local destination of the warp's round-r element (all-ones
// for padding), s_dstart[d] the first destination of digit d and, if non-null,
// dig_count[d] the number of keys with digit d.
struct ChunkRank {
  uint32_t pos[kSegRounds];
};

__device__ __forceinline__ void rank_chunk(const uint32_t* keys, int cnt, int shift, uint32_t* s_w,
                                           uint32_t* s_dstart, uint32_t* s_warp, ChunkRank* cr,
                                           uint32_t* dig_count) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = (cnt + kThreads - 1) / kThreads;
  for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) s_w[d] = 0;
  __syncthreads();
  uint32_t rank[kSegRounds], dig[kSegRounds];
#pragma unroll
  for (int r = 0; r < kSegRounds; ++r) {
    rank[r] = 0;
    dig[r] = 0x100u;
    if (r < R) {
      const int i = warp * 32 * R + r * 32 + lane;
      const bool v = i < cnt;
      const uint32_t d = v ? ((keys[i] >> shift) & 0xFFu) : 0x100u;
      const uint32_t peers = __match_any_sync(kFull, d);
      const uint32_t lt = peers & ((1u << lane) - 1u);
      const uint32_t before = v ? s_w[warp * kRadix + d] : 0u;
      rank[r] = before + __popc(lt);
      dig[r] = d;
      __syncwarp();
      if (v && lt == 0) s_w[warp * kRadix + d] = before + __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t x = s_w[w * kRadix + d];
      s_w[w * kRadix + d] = c;   // exclusive prefix over the warps
      c += x;
    }
    if (dig_count) dig_count[d] = c;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    s_dstart[d] = before + x - c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSegRounds; ++r)
    cr->pos[r] = dig[r] < 0x100u ? s_dstart[dig[r]] + s_w[warp * kRadix + dig[r]] + rank[r]
                                 : 0xFFFFFFFFu;
}

// Runs of equal keys in [0, n) are put in id order (two Gaussians at bit-identical depth
// in one tile).  Each run is handled by the thread at its first element.
__device__ __forceinline__ void order_ties(const uint32_t* keys, uint32_t* ids, int n) {
  for (int i = threadIdx.x; i + 1 < n; i += kThreads) {
    if (keys[i] != keys[i + 1] || (i > 0 && keys[i - 1] == keys[i])) continue;
    int e = i + 1;
    while (e + 1 < n && keys[e + 1] == keys[i]) ++e;
    for (int a = i + 1; a <= e; ++a) {   // insertion sort of ids[i..e]
      const uint32_t v = ids[a];
      int b = a - 1;
      while (b >= i && ids[b] > v) {
        ids[b + 1] = ids[b];
        --b;
      }
      ids[b + 1] = v;
    }
  }
}

// Bits that differ among the block's values: OR ^ AND over the block.
__device__ __forceinline__ uint32_t block_diff_bits(uint32_t v_or, uint32_t v_and, uint32_t* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v_or |= __shfl_xor_sync(kFull, v_or, o);
    v_and &= __shfl_xor_sync(kFull, v_and, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_red[warp] = v_or;
    s_red[kWarps + warp] = v_and;
  }
  __syncthreads();
  uint32_t o = 0, a = 0xFFFFFFFFu;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    o |= s_red[w];
    a &= s_red[kWarps + w];
  }
  __syncthreads();
  return o ^ a;
}

// One block per tile (persistent, heavy-first): sort the tile's range by (depth, id).
// Input: the (key, id) pairs of kv in scatter order; output: the sorted ids in id0 (the
// sorted keys are not written back: nothing reads them).  Ranges longer than kSeg are
// sorted through global memory: the first pass reads the pairs and writes (key0, id0);
// later passes alternate between (key0, id0) and the range's own part of kv, read as n
// keys followed by n ids (its pairs are consumed by the first pass).
// Five blocks per SM (48 registers, no spill; shared memory holds five): the ranking is a
// chain of shared-memory round trips, so resident warps are what hides its latency.
__global__ void __launch_bounds__(kThreads, 5)
k_bin_sort(TileQueue tq, const uint2* __restrict__ ranges, uint2* __restrict__ kv,
           uint32_t* __restrict__ key0, uint32_t* __restrict__ id0) {
  __shared__ uint32_t s_k[2][kSeg], s_v[2][kSeg];
  __shared__ uint32_t s_w[kWarps * kRadix];
  __shared__ uint32_t s_dstart[kRadix], s_run[kRadix], s_cnt[kRadix];
  __shared__ uint32_t s_warp[kWarps], s_red[2 * kWarps];
  __shared__ int s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t q = atomicAdd(tq.head, 1u);
      s_tile = q < (uint32_t)tq.n_tiles ? (int)(tq.order ? tq.order[q] : q) : -1;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) break;
    const uint2 rg = ranges[tile];
    const int s = (int)rg.x, n = (int)(rg.y - rg.x);
    if (n <= 1) {
      if (n == 1 && threadIdx.x == 0) id0[s] = kv[s].y;
      __syncthreads();
      continue;
    }
    if (n <= kSeg) {
      // the pairs into shared memory, and the digit bytes that differ across the range
      // (the others need no pass)
      uint32_t vo = 0, va = 0xFFFFFFFFu;
      for (int i = threadIdx.x; i < n; i += kThreads) {
        const uint2 e = kv[s + i];
        s_k[0][i] = e.x;
        s_v[0][i] = e.y;
        vo |= e.x;
        va &= e.x;
      }
      const uint32_t diff = block_diff_bits(vo, va, s_red);   // (its barrier publishes the chunk)
      int cur = 0;
      const int R = (n + kThreads - 1) / kThreads;
      for (int p = 0; p < 4; ++p) {
        if (((diff >> (8 * p)) & 0xFFu) == 0u) continue;
        ChunkRank cr;
        rank_chunk(s_k[cur], n, 8 * p, s_w, s_dstart, s_warp, &cr, nullptr);
#pragma unroll
        for (int r = 0; r < kSegRounds; ++r) {
          const int i = warp * 32 * R + r * 32 + lane;
          if (r < R && i < n) {
            s_k[cur ^ 1][cr.pos[r]] = s_k[cur][i];
            s_v[cur ^ 1][cr.pos[r]] = s_v[cur][i];
          }
        }
        __syncthreads();
        cur ^= 1;
      }
      order_ties(s_k[cur], s_v[cur], n);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kThreads) id0[s + i] = s_v[cur][i];
    } else {
      uint32_t vo = 0, va = 0xFFFFFFFFu;
      for (int i = threadIdx.x; i < n; i += kThreads) {
        const uint32_t k = kv[s + i].x;
        vo |= k;
        va &= k;
      }
      const uint32_t diff = block_diff_bits(vo, va, s_red);
      // long range: LSD passes through global memory, chunks of kSeg taken in order.
      // Source (ka, ia), null while the data is still in the pairs; destination (kb, ib).
      uint32_t* const wk = reinterpret_cast<uint32_t*>(kv + s);   // the range's part of kv
      uint32_t *ka = nullptr, *ia = nullptr, *kb = key0 + s, *ib = id0 + s;
      for (int p = 0; p < 4; ++p) {
        if (((diff >> (8 * p)) & 0xFFu) == 0u) continue;
        // digit histogram of the whole range -> running output offsets per digit
        s_cnt[threadIdx.x] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kThreads)
          atomicAdd(&s_cnt[((ka ? ka[i] : kv[s + i].x) >> (8 * p)) & 0xFFu], 1u);
        __syncthreads();
        {   // exclusive scan of the 256 digit counts, one per thread
          const uint32_t c = s_cnt[threadIdx.x];
          uint32_t x = c;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
          }
          if (lane == 31) s_warp[warp] = x;
          __syncthreads();
          uint32_t before = 0;
          for (int w = 0; w < warp; ++w) before += s_warp[w];
          s_run[threadIdx.x] = before + x - c;
        }
        __syncthreads();
        for (int c0 = 0; c0 < n; c0 += kSeg) {
          const int cnt = min(kSeg, n - c0);
          for (int i = threadIdx.x; i < cnt; i += kThreads) {
            if (ka) {
              s_k[0][i] = ka[c0 + i];
              s_v[0][i] = ia[c0 + i];
            } else {
              const uint2 e = kv[s + c0 + i];
              s_k[0][i] = e.x;
              s_v[0][i] = e.y;
            }
          }
          __syncthreads();
          ChunkRank cr;
          rank_chunk(s_k[0], cnt, 8 * p, s_w, s_dstart, s_warp, &cr, s_cnt);
          const int R = (cnt + kThreads - 1) / kThreads;
#pragma unroll
          for (int r = 0; r < kSegRounds; ++r) {
            const int i = warp * 32 * R + r * 32 + lane;
            if (r < R && i < cnt) {
              const uint32_t d = (s_k[0][i] >> (8 * p)) & 0xFFu;
              const uint32_t o = s_run[d] + (cr.pos[r] - s_dstart[d]);
              kb[o] = s_k[0][i];
              ib[o] = s_v[0][i];
            }
          }
          __syncthreads();
          s_run[threadIdx.x] += s_cnt[threadIdx.x];
          __syncthreads();
        }
        // the next pass reads what this one wrote and writes the other buffer
        const bool to_wk = kb == key0 + s;
        ka = kb;
        ia = ib;
        kb = to_wk ? wk : key0 + s;
        ib = to_wk ? wk + n : id0 + s;
      }
      if (!ka) {   // every key equal: unpack the pairs for the tie order
        for (int i = threadIdx.x; i < n; i += kThreads) {
          const uint2 e = kv[s + i];
          key0[s + i] = e.x;
          id0[s + i] = e.y;
        }
        __syncthreads();
        ka = key0 + s;
        ia = id0 + s;
      }
      order_ties(ka, ia, n);
      __syncthreads();
      if (ia != id0 + s)
        for (int i = threadIdx.x; i < n; i += kThreads) id0[s + i] = ia[i];
    }
    __syncthreads();   // shared memory and s_tile are reused by the next tile
  }
  if (threadIdx.x == 0) queue_leave(tq, gridDim.x);
}

// ---------------------------------------------------------------- statistics

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
  eval = __reduce_add_sync(kFull, eval);
  blend = __reduce_add_sync(kFull, blend);
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
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
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

bool launch_bin(const BinArgs& b, cudaStream_t st) {
  const int T = b.n_tiles;
  if (T <= 0) return false;
  const unsigned gb = (unsigned)max64(ceil_div(b.n, kThreads), 1);
  uint32_t* order = T <= kMaxOrderedTiles ? b.order : nullptr;
  if (count_tile_rows(T)) {   // the projection left per-row differences
    const int TY = T / b.TX;
    k_bin_rows<<<(unsigned)ceil_div(TY, kWarps), kThreads, 0, st>>>(b.tile_count, b.TX, TY);
    note_launch();
  }
  k_bin_scan<<<1, kScanThreads, 0, st>>>(b.tile_count, T, b.TX, b.cap, b.ranges, b.cursor, order,
                                         b.counters);
  note_launch();
  if (b.n > 0) {
    k_bin_scatter<<<gb, kThreads, 0, st>>>(b.n, b.ntiles, b.rect, b.depth_key, b.TX, T, b.cap,
                                           b.cursor, b.kv);
    note_launch();
  }
  // per-tile sort: persistent blocks over the tiles, heaviest first
  const TileQueue tq{b.queue, b.queue + 1, order, T};
  const int grid = persistent_grid(k_bin_sort, kThreads, 0, T);
  k_bin_sort<<<grid, kThreads, 0, st>>>(tq, b.ranges, b.kv, b.key0, b.id0);
  note_launch();
  return order != nullptr;
}

void launch_pair_stats(const CamDev& cam, const GaussRec* rec, const uint2* ranges,
                       const uint32_t* inst_id, const uint32_t* n_contrib,
                       unsigned long long* stats64, cudaStream_t st) {
  cudaMemsetAsync(stats64, 0, 2 * sizeof(unsigned long long), st);
  if (cam.TX * cam.TY == 0) return;
  k_pair_stats<<<cam.TX * cam.TY, kThreads, 0, st>>>(cam, rec, ranges, inst_id, n_contrib, stats64);
  note_launch();
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
