// Workspace operations of the serving executor (gs_serve.cu), implemented in gs_api.cu;
// host-only, outside the C ABI.
#pragma once

#include "gs_internal.cuh"

namespace gs {
gs_status ws_reserve_fixed(gs_workspace* ws, int64_t n_gauss, int64_t n_pixels, int64_t n_tiles);
// The instance buffers become the caller's ranges (cap slots each: (key, id) pairs, scratch
// keys, sorted ids; not freed by the workspace).
void ws_lend_instances(gs_workspace* ws, uint2* kv, uint32_t* key0, uint32_t* id0, int64_t cap);
bool ws_fits(const gs_workspace* ws, int64_t n_gauss, int64_t n_pixels, int64_t n_tiles);
// Asynchronous copy of the projection's tile-instance count to *host (pinned).
gs_status ws_instances_async(gs_workspace* ws, uint32_t* host, cudaStream_t st);
// Raster job of the workspace's binned render of sc (outputs and gradients left null).
gs_status ws_job(gs_workspace* ws, const gs_scene& sc, RasterJob* job);
int ws_tiles(const gs_workspace* ws);
// Zeroes the backward accumulators (and g_feats) before a backward raster launch.
gs_status ws_bwd_clear(gs_workspace* ws, int D, float* g_feats, cudaStream_t st);
gs_status ws_project_bwd(gs_workspace* ws, const gs_scene& sc, float* g_means, float* g_scales,
                         float* g_quats, float* g_opac, float* g_sh, float* g_pose6, cudaStream_t st);

}  // namespace gs
