// Per-(pixel, Gaussian) opacity evaluation shared by the forward and backward raster
// kernels.  Both kernels must take identical skip decisions for a pixel, so the
// arithmetic is pinned with explicit rounding intrinsics (no contraction freedom).
#pragma once

#include <cuda_runtime.h>

namespace gs {

constexpr float kAlphaMin = 1.f / 255.f;   // skip a Gaussian with alpha below this
constexpr float kAlphaMax = 0.99f;         // alpha cap
constexpr float kTMin = 1e-4f;             // stop before T would drop below this

// sigma = 1/2 (A dx^2 + C dy^2) + B dx dy for the offset (dx, dy) = pixel - mean
// (the exponent of G(x), App. A, with the 2D conic [[A, B], [B, C]]).
__device__ __forceinline__ float blend_sigma(float dx, float dy, float A, float B, float C) {
  const float q = __fmaf_rn(__fmul_rn(C, dy), dy, __fmul_rn(__fmul_rn(A, dx), dx));
  return __fmaf_rn(0.5f, q, __fmul_rn(__fmul_rn(B, dx), dy));
}

// G = exp(-sigma) and o*G; the caller applies the cap and thresholds.
__device__ __forceinline__ float blend_gauss(float sigma) { return __expf(-sigma); }

}  // namespace gs
