// Grid-sampled supervision targets (X-GS Sec. 3.2 and App. D): the target map G* and the
// validity mask V on the same compact stride-s grid the renderer draws, from either a
// segmentation with a region-feature table or a lower-resolution continuous feature map.
// One thread per sample; each thread writes its D channels (channel-major output, so a
// warp's stores of one channel are contiguous).
#include <cstdint>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

// Region-indexed: V = [S(u, v) in [0, R)], G* = Phi[S(u, v)] where valid, else 0.
__global__ void __launch_bounds__(kThreads)
k_target_region(const int32_t* __restrict__ seg, int H, int W, const float* __restrict__ table,
                int R, int D, int s, int ox, int oy, int Hs, int Ws, float* __restrict__ target,
                float* __restrict__ mask) {
  const int64_t HsWs = (int64_t)Hs * Ws;
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= HsWs) return;
  const int m = (int)(p / Ws), n = (int)(p - (int64_t)m * Ws);
  const int u = grid_coord(oy, s, m), v = grid_coord(ox, s, n);
  int sid = -1;
  if (u < H && v < W) sid = seg[(int64_t)u * W + v];
  const bool ok = sid >= 0 && sid < R;
  if (mask) mask[p] = ok ? 1.f : 0.f;
  if (ok) {
    const float* row = table + (int64_t)sid * D;
    for (int c = 0; c < D; ++c) target[c * HsWs + p] = __ldg(row + c);
  } else {
    for (int c = 0; c < D; ++c) target[c * HsWs + p] = 0.f;
  }
}

// round(num / den) for num >= 0, den > 0, halves away from zero, exactly.
__device__ __forceinline__ int64_t round_ratio(int64_t num, int64_t den) {
  return (2 * num + den) / (2 * den);
}

// Continuous map: u~ = round(u (Hf - 1) / max(H - 1, 1)), v~ likewise; V = 1 inside the
// image, 0 for samples beyond it.
__global__ void __launch_bounds__(kThreads)
k_target_resample(const float* __restrict__ fmap, int D, int Hf, int Wf, int H, int W, int s,
                  int ox, int oy, int Hs, int Ws, float* __restrict__ target,
                  float* __restrict__ mask) {
  const int64_t HsWs = (int64_t)Hs * Ws;
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= HsWs) return;
  const int m = (int)(p / Ws), n = (int)(p - (int64_t)m * Ws);
  const int u = grid_coord(oy, s, m), v = grid_coord(ox, s, n);
  const bool ok = u < H && v < W;
  if (mask) mask[p] = ok ? 1.f : 0.f;
  if (ok) {
    // u <= H - 1 gives u~ <= Hf - 1 (and likewise v~): always inside the map
    const int64_t uu = round_ratio((int64_t)u * (Hf - 1), H > 1 ? H - 1 : 1);
    const int64_t vv = round_ratio((int64_t)v * (Wf - 1), W > 1 ? W - 1 : 1);
    const int64_t HfWf = (int64_t)Hf * Wf;
    const float* src = fmap + uu * Wf + vv;
    for (int c = 0; c < D; ++c) target[c * HsWs + p] = __ldg(src + c * HfWf);
  } else {
    for (int c = 0; c < D; ++c) target[c * HsWs + p] = 0.f;
  }
}

bool grid_args_ok(int H, int W, int s, int ox, int oy) {
  return H > 0 && W > 0 && s >= 1 && s <= kMaxStride && ox >= 0 && ox < s && oy >= 0 && oy < s;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_grid_target_region(const int32_t* seg, int32_t H, int32_t W, const float* table,
                                int32_t R, int32_t D, int32_t stride, int32_t off_x, int32_t off_y,
                                float* target, float* mask, void* stream) {
  if (!grid_args_ok(H, W, stride, off_x, off_y) || R < 0 || D < 0 || !seg ||
      (D > 0 && (!target || (R > 0 && !table))))
    return GS_ERR_ARG;
  const int Hs = (H + stride - 1) / stride, Ws = (W + stride - 1) / stride;
  const int64_t P = (int64_t)Hs * Ws;
  k_target_region<<<(unsigned)ceil_div(P, kThreads), kThreads, 0, (cudaStream_t)stream>>>(
      seg, H, W, table, R, D, stride, off_x, off_y, Hs, Ws, target, mask);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_grid_target_resample(const float* fmap, int32_t D, int32_t Hf, int32_t Wf, int32_t H,
                                  int32_t W, int32_t stride, int32_t off_x, int32_t off_y,
                                  float* target, float* mask, void* stream) {
  if (!grid_args_ok(H, W, stride, off_x, off_y) || D < 0 || Hf <= 0 || Wf <= 0 ||
      (D > 0 && (!fmap || !target)))
    return GS_ERR_ARG;
  const int Hs = (H + stride - 1) / stride, Ws = (W + stride - 1) / stride;
  const int64_t P = (int64_t)Hs * Ws;
  k_target_resample<<<(unsigned)ceil_div(P, kThreads), kThreads, 0, (cudaStream_t)stream>>>(
      fmap, D, Hf, Wf, H, W, stride, off_x, off_y, Hs, Ws, target, mask);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
