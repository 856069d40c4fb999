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
// Also adds V (visible Gaussians) and I (tile instances) to counters[kCntVisible/kCntInst].
void launch_project(const gs_scene& sc, const CamDev& cam, GaussRec* rec, uint32_t* depth_key,
                    uint32_t* ntiles, uint2* rect, uint32_t* counters, cudaStream_t st);

// gs_sort.cu: binning in tile buckets (count, scan, scatter, per-tile radix sort).
// After launch_bin, tile t's Gaussians occupy slots [ranges[t].x, ranges[t].y) of id0 in
// (depth, id) order (key0 holds their depth keys, tile_out their tile); slots are capped
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
  uint32_t* tile_count;          // [n_tiles] scratch
  uint32_t* cursor;              // [n_tiles] scratch
  uint2* ranges;                 // [n_tiles] out
  uint32_t* order;               // [n_tiles] out (heavy-first)
  uint32_t* queue;               // one word (persistent sort queue head)
  uint32_t *key0, *id0;          // [cap] out: sorted depth keys and Gaussian ids
  uint32_t *key1, *id1;          // [cap] scratch (ranges longer than shared memory)
  uint32_t* tile_out;            // [cap] out: tile of every slot
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

// Persistent raster scheduling: a CTA takes the next tile index from *queue (zeroed
// before each launch) and maps it through `order` (identity when null).
struct TileQueue {
  uint32_t* head;
  const uint32_t* order;
  int n_tiles;
};

// Grid of a persistent kernel: as many CTAs as fit on the device at once (never more than
// n_items).  Sets the kernel's dynamic shared-memory limit to `smem`: static plus dynamic
// shared memory above 48 KB needs it even when the dynamic part alone is below 48 KB.
template <class Kernel>
inline int persistent_grid(Kernel kern, int threads, size_t smem, int n_items) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  const int g = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return n_items < g ? (n_items > 0 ? n_items : 1) : g;
}

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

// gs_raster_bwd.cu
// Accumulators per Gaussian: g2d[12*i + k], k = u, v, A, B, C, o, r, g, b, z
constexpr int kG2D = 12;
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
