// Internal declarations shared by the CUDA translation units of libgs.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kTile = 16;
constexpr int kTilePix = kTile * kTile;   // 256 pixels, one thread each
constexpr int kMaxFeat = 64;
constexpr int kMaxStride = 256;   // largest sample-grid stride

// Per-Gaussian record written by the projection and gathered by the rasterizer:
// r0 = (u, v, A, B), r1 = (C, opacity, depth, 0), r2 = (r, g, b, 0); 48 bytes.
// (u, v) is the 2D mean in pixels, (A, B, C) the conic [[A, B], [B, C]] = Sigma'^-1.
struct __align__(16) GaussRec {
  float4 r0, r1, r2;
};

// Camera as the kernels see it.  W, H, TX, TY are the image and its 16x16 tiles, in which
// Gaussians are always binned.  The rendered pixels are the image itself (stride 1) or,
// for grid-sampled supervision (App. D), the compact GW x GH grid whose sample (n, m) is
// image pixel (ox + n s, oy + m s).
struct CamDev {
  int W, H, TX, TY;
  int n_gauss;   // number of Gaussians (bounds check of gathered ids)
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float near_z;
  int stride, ox, oy;
  int GW, GH;
};

// Image pixel coordinate of compact sample index k along an axis with offset o.
__host__ __device__ inline int grid_coord(int o, int stride, int k) { return o + k * stride; }

// Device status word bits.
enum : uint32_t {
  kErrInstOverflow = 1u,   // instance count above reserved capacity (no-sync binning)
  kErrBadRange = 2u,       // a tile range outside the instance array (guard)
};

// Device counters (one small array in the workspace).
enum : int {
  kCntVisible = 0,   // V
  kCntInst = 1,      // I (true count, may exceed capacity)
  kCntStatus = 2,    // status word
  kCntInstEff = 3,   // I_eff (stats)
  kCntNum = 8
};

// ---- launchers (each .cu file defines its own) --------------------------------------

// gs_project_fwd.cu
// Also adds V (visible Gaussians) and I (tile instances) to counters[kCntVisible/kCntInst]
// and each Gaussian's tiles to tile_count[cam.TX * cam.TY] (the binning's per-tile counts,
// zero before the launch; the binning's scan clears them again after reading them).
void launch_project(const gs_scene& sc, const CamDev& cam, GaussRec* rec, uint32_t* depth_key,
                    uint32_t* ntiles, uint2* rect, uint32_t* counters, uint32_t* tile_count,
                    cudaStream_t st);

// gs_sort.cu: binning in tile buckets (scan, scatter, per-tile radix sort; the count is
// added by the projection).  After launch_bin, tile t's Gaussians occupy slots [ranges[t].x, ranges[t].y) of id0 in
// (depth, id) order (kv holds the scattered (key, id) pairs; kv and key0 are also scratch); slots are capped
// at `cap` (an instance count above it sets kErrInstOverflow).  `order` receives the
// heavy-first tile order when there are at most kMaxOrderedTiles tiles (the return value
// says whether it was written).  No host synchronisation.
struct BinArgs {
  int64_t n;                     // Gaussians
  const uint32_t* ntiles;        // [n] tiles per Gaussian (0 = culled)
  const uint2* rect;             // [n] packed tile rectangles
  const uint32_t* depth_key;     // [n]
  int TX, n_tiles;
  int64_t cap;                   // instance slots available
  uint32_t* tile_count;          // [TY (TX + 1)] per-row tile count differences (from the
                                 // projection; the row pass and the scan zero them)
  uint32_t* cursor;              // [n_tiles] scratch
  uint2* ranges;                 // [n_tiles] out
  uint32_t* order;               // [n_tiles] out (heavy-first)
  uint32_t* queue;               // two words: the persistent sort's queue head and leave count
  uint2* kv;                     // [cap] (depth key, id) pairs of the scatter
  uint32_t *key0, *id0;          // [cap] id0 out: sorted Gaussian ids; key0: scratch (ranges
                                 // longer than shared memory)
  uint32_t* counters;            // workspace counters (status word)
};
constexpr int kMaxOrderedTiles = 1 << 18;
bool launch_bin(const BinArgs& b, cudaStream_t st);
void launch_inst_eff(const uint32_t* n_contrib, int TX, int TY, int W, int H, uint32_t* counters,
                     cudaStream_t st);
// Pair counts for the roofline model (stats only): stats64[0] = evaluated, [1] = blended.
void launch_pair_stats(const CamDev& cam, const GaussRec* rec, const uint2* ranges,
                       const uint32_t* inst_id, const uint32_t* n_contrib,
                       unsigned long long* stats64, cudaStream_t st);

// Persistent raster scheduling: a CTA (or warp) takes the next item index from *head and
// maps it through `order` (identity when null).  The forward, sort and grid-forward queues
// reset themselves: every participant calls queue_leave() once after its last take, and
// the last one to leave puts head and done back to zero, so a launch finds both at zero
// without a memset (they are zeroed once when allocated).  The backward kernels' queue is
// zeroed by the host before each launch.
struct TileQueue {
  uint32_t* head;
  uint32_t* done;
  const uint32_t* order;
  int n_tiles;
};

// The tile instances of the 32 Gaussians of a warp, flattened: instance k of the warp
// (Gaussians in lane order, tiles of a Gaussian in row-major order of its rectangle).
// warp_instances_begin takes the calling lane's tile count nt and packed rectangle rc
// (x0 | y0 << 16, x1 | y1 << 16); warp_instance_tile returns the tile of instance k
// (0xFFFFFFFF for k >= total) and its owner lane.  Every lane of the warp must call both.
struct WarpInstances {
  uint32_t excl, total;
  uint2 rc;
};
__device__ __forceinline__ WarpInstances warp_instances_begin(uint32_t nt, uint2 rc) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = nt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  return WarpInstances{incl - nt, __shfl_sync(0xffffffffu, incl, 31), rc};
}
__device__ __forceinline__ uint32_t warp_instance_tile(const WarpInstances& wi, uint32_t k, int TX,
                                                       int* owner) {
  const unsigned full = 0xffffffffu;
  // owner: the last lane whose first instance is <= k (it has at least one instance)
  int lo = 0, hi = 31;
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    const int mid = (lo + hi + 1) >> 1;
    const uint32_t e = __shfl_sync(full, wi.excl, mid);
    if (e <= k) lo = mid; else hi = mid - 1;
  }
  const uint32_t oe = __shfl_sync(full, wi.excl, lo);
  const uint32_t rx = __shfl_sync(full, wi.rc.x, lo), ry = __shfl_sync(full, wi.rc.y, lo);
  uint32_t tile = 0xFFFFFFFFu;
  if (k < wi.total) {
    const uint32_t x0 = rx & 0xFFFFu, y0 = rx >> 16, w = (ry & 0xFFFFu) - x0;
    const uint32_t q = k - oe;
    if (w) tile = (y0 + q / w) * (uint32_t)TX + x0 + q % w;
  }
  *owner = lo;
  return tile;
}

// Calls f(owner_lane, tile) for the warp's instances, 32 per round (lane j takes instance
// round * 32 + j; tile = 0xFFFFFFFF past the last); every lane calls it in every round.
template <class F>
__device__ __forceinline__ void warp_tile_instances(uint32_t nt, uint2 rc, int TX, F f) {
  const WarpInstances wi = warp_instances_begin(nt, rc);
  for (uint32_t base = 0; base < wi.total; base += 32) {
    int lo;
    const uint32_t tile = warp_instance_tile(wi, base + (threadIdx.x & 31), TX, &lo);
    f(lo, tile);
  }
}

// Slot of tile i (row-major, TX tiles per row) in the binning's per-tile count array,
// which holds TY rows of TX + 1 words: the projection adds row differences there, and the
// binning's row pass turns each row into counts in place (the last word of a row is the
// difference past the right edge).
__device__ __forceinline__ uint32_t tile_slot(uint32_t i, int TX) { return i + i / (uint32_t)TX; }

// The count step's form, the same on the host and in the kernels: frames of at least 4096
// tiles (Gaussians covering many tiles) add per-row differences (warp_count_rows, then the
// binning's row pass); smaller frames add per-tile counts at tile_slot (warp_count_tiles,
// merged within a warp) and need no row pass.
constexpr int kRowCountTiles = 4096;
__host__ __device__ inline bool count_tile_rows(int n_tiles) { return n_tiles >= kRowCountTiles; }

// Adds each lane's tile instances at tile_slot: one atomic per distinct tile per warp round.
__device__ __forceinline__ void warp_count_tiles(uint32_t nt, uint2 rc, int TX, int n_tiles,
                                                 uint32_t* tile_count) {
  warp_tile_instances(nt, rc, TX, [&](int, uint32_t tile) {
    const bool ok = tile < (uint32_t)n_tiles;
    const uint32_t peers = __match_any_sync(0xffffffffu, ok ? tile : 0xFFFFFFFFu);
    if (ok && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0)
      atomicAdd(&tile_count[tile_slot(tile, TX)], (uint32_t)__popc(peers));
  });
}

// Adds each lane's tile rectangle to the per-row difference array: +1 at its first tile
// and -1 past its last tile of every tile row it covers (two atomics per row; the row
// pass of the binning sums them into per-tile counts).  The warp's rows are flattened
// across its lanes, 32 per round.
__device__ __forceinline__ void warp_count_rows(uint32_t nt, uint2 rc, int TX, uint32_t* tile_diff) {
  const uint32_t x0 = rc.x & 0xFFFFu, y0 = rc.x >> 16, x1 = rc.y & 0xFFFFu, y1 = rc.y >> 16;
  const uint32_t rows = nt ? y1 - y0 : 0u;
  const WarpInstances wi = warp_instances_begin(rows, rc);
  const unsigned full = 0xffffffffu;
  const uint32_t stride = (uint32_t)TX + 1u;
  for (uint32_t base = 0; base < wi.total; base += 32) {
    const uint32_t k = base + (threadIdx.x & 31);
    // owner: the last lane whose first row is <= k (it has at least one row)
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (lo + hi + 1) >> 1;
      const uint32_t e = __shfl_sync(full, wi.excl, mid);
      if (e <= k) lo = mid; else hi = mid - 1;
    }
    const uint32_t oe = __shfl_sync(full, wi.excl, lo);
    const uint32_t rx = __shfl_sync(full, rc.x, lo), ry = __shfl_sync(full, rc.y, lo);
    if (k < wi.total) {
      const uint32_t row = (rx >> 16) + (k - oe);
      atomicAdd(&tile_diff[row * stride + (rx & 0xFFFFu)], 1u);
      atomicAdd(&tile_diff[row * stride + (ry & 0xFFFFu)], 0xFFFFFFFFu);   // -1
    }
  }
}

__device__ __forceinline__ void queue_leave(const TileQueue& tq, unsigned participants) {
  __threadfence();   // this participant's takes precede its leave
  if (atomicAdd(tq.done, 1u) == participants - 1u) {
    atomicExch(tq.head, 0u);
    atomicExch(tq.done, 0u);
  }
}

// Resident CTAs of a kernel on the current device (SMs x CTAs per SM), computed once per
// (kernel, block size, dynamic shared memory, device) and cached: the attribute and
// occupancy queries cost host time on every launch otherwise.  Sets the kernel's dynamic
// shared-memory limit to `smem` on first use: static plus dynamic shared memory above 48 KB
// needs it even when the dynamic part alone is below 48 KB.
int resident_ctas(const void* kern, int threads, size_t smem);

// Grid of a persistent kernel: as many CTAs as fit on the device at once (never more than
// n_items).
template <class Kernel>
inline int persistent_grid(Kernel kern, int threads, size_t smem, int n_items) {
  const int g = resident_ctas(reinterpret_cast<const void*>(kern), threads, smem);
  return n_items < g ? (n_items > 0 ? n_items : 1) : g;
}

// One render in a raster launch: its camera, inputs and outputs.  A launch takes a table of
// up to NJ of them and drains their work items through one persistent grid (serving batches
// several requests' tiles into one launch this way; a plain render is a table of one).  Work
// items of job k are [job[k-1].item_end, job[k].item_end) of the launch's queue, taken in
// the job's heavy-first tile order.
struct RasterJob {
  CamDev cam;
  const GaussRec* rec;
  const void* feats;
  int D;
  int item_end;
  const uint2* ranges;
  const uint32_t* inst_id;
  const uint32_t* order;        // heavy-first tile order, or null (row-major)
  float *rgb, *depth, *alpha, *feat;   // forward outputs (any may be null)
  float* T_final;               // written by the forward, read by the backward
  uint32_t* n_contrib;
  const float *g_rgb, *g_depth, *g_alpha, *g_feat;   // backward inputs
  float *g2d, *g_feats;         // backward accumulators
};
constexpr int kMaxJobs = 8;
template <int NJ>
struct RasterJobs {
  int n;
  RasterJob job[NJ];
  // job of work item q (q below the last item_end) and the first item of that job
  __device__ __forceinline__ int find(uint32_t q, uint32_t* first) const {
    int k = 0;
    if constexpr (NJ > 1)
      while (k < n - 1 && q >= (uint32_t)job[k].item_end) ++k;
    *first = k > 0 ? (uint32_t)job[k - 1].item_end : 0u;
    return k;
  }
  __device__ __forceinline__ uint32_t items() const { return (uint32_t)job[NJ > 1 ? n - 1 : 0].item_end; }
};

// gs_raster_fwd.cu
// Masked L1 + cosine feature loss (App. D) fused into the forward's epilogue; inactive
// when target is null.  Per sample p with a = V_p G_hat[:, p], b = V_p G*[:, p]:
// L_1 = sum |a - b| / (D P), L_cos = sum_p (1 - cos(a, b)) / P, L = lambda (L_1 + L_cos).
struct FeatLoss {
  const float* target;   // G* [D][GH][GW]
  const float* mask;     // V [GH][GW]; null = all ones
  float* g_feat;         // out: dL/dG_hat [D][GH][GW]
  double* loss;          // out: L, L_1, L_cos (accumulated; zeroed by the caller)
  float w_l1, w_cos;     // lambda / (D P), lambda / P
  double s_l1, s_cos, lambda;   // 1 / (D P), 1 / P, lambda
};
constexpr float kCosEps = 1e-8f;

// loss: the fused feature loss, or null.
void launch_raster_fwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec,
                       const void* feats, int feat_dtype, int D, const uint2* ranges,
                       const uint32_t* inst_id, float* rgb, float* depth, float* alpha, float* feat,
                       float* T_final, uint32_t* n_contrib, const FeatLoss* loss,
                       cudaStream_t st);

// Forward raster of a table of n <= kMaxJobs jobs that share one feature layout (padded
// channel count and dtype) in one persistent launch; item_end counts half tiles (two per
// tile).  No fused loss.
void launch_raster_fwd_jobs(const RasterJob* jobs, int n, int feat_dtype, bool want_feat,
                            const TileQueue& tq, cudaStream_t st);
// Half-tile work items of the forward per tile.
constexpr int kFwdItemsPerTile = 2;

// gs_raster_bwd.cu
// Accumulators per Gaussian: g2d[12*i + k], k = u, v, A, B, C, o, r, g, b, z
constexpr int kG2D = 12;
// Backward raster of a table of n <= kMaxJobs jobs (every gradient; item_end counts tiles;
// the queue is zeroed by the caller).
void launch_raster_bwd_jobs(const RasterJob* jobs, int n, int feat_dtype, bool want_feat,
                            const TileQueue& tq, cudaStream_t st);
void launch_raster_bwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec,
                       const void* feats, int feat_dtype,
                       int D, const uint2* ranges, const uint32_t* inst_id, const float* T_final,
                       const uint32_t* n_contrib, const float* g_rgb, const float* g_depth,
                       const float* g_alpha, const float* g_feat, float* g2d, float* g_feats,
                       bool features_only, cudaStream_t st);

// gs_raster_grid.cu: rendering on a stride-s sample grid (stride > 1), one warp per work
// item = (image tile, chunk of up to 32 of the tile's samples), over the image-tile lists.
int grid_chunks_per_tile(int stride);
void launch_grid_fwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec, const void* feats,
                     int feat_dtype, int D, const uint2* ranges, const uint32_t* inst_id, float* rgb,
                     float* depth, float* alpha, float* feat, float* T_final, uint32_t* n_contrib,
                     const FeatLoss* loss, cudaStream_t st);
void launch_grid_bwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec, const void* feats,
                     int feat_dtype, int D, const uint2* ranges, const uint32_t* inst_id,
                     const float* T_final, const uint32_t* n_contrib, const float* g_rgb,
                     const float* g_depth, const float* g_alpha, const float* g_feat, float* g2d,
                     float* g_feats, bool features_only, cudaStream_t st);
// Pair counts and I_eff (sum over work items of the longest list prefix) of a grid render.
void launch_grid_stats(const CamDev& cam, const GaussRec* rec, const uint2* ranges,
                       const uint32_t* inst_id, const uint32_t* n_contrib, uint32_t* item_max,
                       uint32_t* counters, unsigned long long* stats64, cudaStream_t st);

// gs_project_bwd.cu
int project_bwd_blocks(int64_t n);
void launch_project_bwd(const gs_scene& sc, const CamDev& cam, const GaussRec* rec,
                        const uint32_t* ntiles, const float* g2d, float* g_means, float* g_scales,
                        float* g_quats, float* g_opac, float* g_sh, float* pose_partials,
                        float* g_pose6, cudaStream_t st);
void launch_l1_grad(const float* pred, const float* target, int64_t n, float scale, float* grad,
                    cudaStream_t st);

int padded_feat(int D);

// Count kernels launched by the library (process-wide; read with gs_launch_count()).
void note_launch(int k = 1);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

}  // namespace gs
