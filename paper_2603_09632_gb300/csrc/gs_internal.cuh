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

// Per-Gaussian record written by the projection and gathered by the rasterizer:
// r0 = (u, v, A, B), r1 = (C, opacity, depth, 0), r2 = (r, g, b, 0); 48 bytes.
// (u, v) is the 2D mean in pixels, (A, B, C) the conic [[A, B], [B, C]] = Sigma'^-1.
struct __align__(16) GaussRec {
  float4 r0, r1, r2;
};

// Camera as the kernels see it.
struct CamDev {
  int W, H, TX, TY;
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float near_z;
};

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
void launch_project(const gs_scene& sc, const CamDev& cam, GaussRec* rec, uint32_t* depth_key,
                    uint32_t* ntiles, uint2* rect, cudaStream_t st);

// gs_sort.cu
size_t scan_temp_words(int64_t n);
// exclusive scan of n u32 (n known on the host); in may equal out
void device_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* temp,
                           cudaStream_t st);
// number of histogram words the radix sort needs for `bound` elements
size_t radix_hist_words(int64_t bound);
// Stable LSD radix sort of (key, val) pairs over key bits [0, end_bit).  The element count
// is *d_n (device), at most `bound` (host).  Ping-pongs between (k0,v0) and (k1,v1);
// returns 0 if the result is in (k0, v0), 1 if in (k1, v1).
int radix_sort_pairs(const uint32_t* d_n, int64_t bound, uint32_t* k0, uint32_t* v0,
                     uint32_t* k1, uint32_t* v1, int end_bit, uint32_t* hist,
                     uint32_t* scan_temp, cudaStream_t st);
// visible compaction: ids and depth keys of Gaussians with ntiles > 0, in id order;
// writes V to counters[kCntVisible].
void launch_compact_visible(const uint32_t* ntiles, const uint32_t* depth_key, int64_t n,
                            uint32_t* flags_scan, uint32_t* out_keys, uint32_t* out_ids,
                            uint32_t* counters, uint32_t* scan_temp, cudaStream_t st);
// per visible Gaussian in depth order: tile count -> exclusive offsets; I -> counters.
void launch_tile_offsets(const uint32_t* sorted_ids, const uint32_t* ntiles, int64_t bound_v,
                         uint32_t* counters, uint32_t* offsets, uint32_t* scan_temp,
                         cudaStream_t st);
// emit (tile, id) instances in depth order, at most cap (overflow flagged)
void launch_emit_instances(const uint32_t* sorted_ids, const uint2* rect, const uint32_t* offsets,
                           int64_t bound_v, int TX, uint32_t* counters, int64_t cap,
                           uint32_t* inst_tile, uint32_t* inst_id, cudaStream_t st);
// tile ranges [start, end) from tile-sorted instances
void launch_tile_ranges(const uint32_t* inst_tile, const uint32_t* counters, int64_t bound_i,
                        int64_t cap, int n_tiles, uint2* ranges, cudaStream_t st);
void launch_inst_eff(const uint2* ranges, const uint32_t* n_contrib, int TX, int TY, int W, int H,
                     uint32_t* counters, cudaStream_t st);

// gs_raster_fwd.cu
void launch_raster_fwd(const CamDev& cam, const GaussRec* rec, const void* feats, int feat_dtype,
                       int D, const uint2* ranges, const uint32_t* inst_id, float* rgb,
                       float* depth, float* alpha, float* feat, float* T_final,
                       uint32_t* n_contrib, cudaStream_t st);

// gs_raster_bwd.cu
// Accumulators per Gaussian: g2d[12*i + k], k = u, v, A, B, C, o, r, g, b, z
constexpr int kG2D = 12;
void launch_raster_bwd(const CamDev& cam, const GaussRec* rec, const void* feats, int feat_dtype,
                       int D, const uint2* ranges, const uint32_t* inst_id, const float* T_final,
                       const uint32_t* n_contrib, const float* g_rgb, const float* g_depth,
                       const float* g_alpha, const float* g_feat, float* g2d, float* g_feats,
                       cudaStream_t st);

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
