// Per-(pixel, Gaussian) opacity evaluation shared by the forward and backward raster
// kernels.  Both kernels must take identical skip decisions for a pixel, so the
// arithmetic is pinned with explicit rounding intrinsics (no contraction freedom).
#pragma once

#include <cuda_runtime.h>

namespace gs {

constexpr float kAlphaMin = 1.f / 255.f;   // skip a Gaussian with alpha below this
constexpr float kAlphaMax = 0.99f;         // alpha cap
constexpr float kTMin = 1e-4f;             // stop before T would drop below this

// Two FP32 fused multiply-adds (or products) in one packed instruction of the sm_100
// family.  Each component is rounded exactly as fmaf (or __fmul_rn), so a sum accumulated
// in packed pairs equals the scalar one bit for bit; the raster kernels are bound by
// instruction issue, and the packed form halves the issue slots of their accumulations.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 splat2(float x) { return make_float2(x, x); }
// component c of a vector held as packed pairs
__device__ __forceinline__ float pair_at(const float2* v, int c) { return (c & 1) ? v[c >> 1].y : v[c >> 1].x; }

// sigma = 1/2 (A dx^2 + C dy^2) + B dx dy for the offset (dx, dy) = pixel - mean
// (the exponent of G(x), App. A, with the 2D conic [[A, B], [B, C]]).
__device__ __forceinline__ float blend_sigma(float dx, float dy, float A, float B, float C) {
  const float q = __fmaf_rn(__fmul_rn(C, dy), dy, __fmul_rn(__fmul_rn(A, dx), dx));
  return __fmaf_rn(0.5f, q, __fmul_rn(__fmul_rn(B, dx), dy));
}

// G = exp(-sigma) and o*G; the caller applies the cap and thresholds.
__device__ __forceinline__ float blend_gauss(float sigma) { return __expf(-sigma); }

// sigma at offset dx (fixed) minimised over dy in [lo, hi] (convex quadratic in dy).
__device__ __forceinline__ float edge_min_sigma(float dx, float lo, float hi, float a, float b,
                                                float c) {
  const float dy = fminf(fmaxf(-b * dx / c, lo), hi);
  return 0.5f * (a * dx * dx + c * dy * dy) + b * dx * dy;
}

// sigma above which a pixel cannot reach alpha >= 1/255: ln(255 o) plus a margin of 1e-3
// (0.1 % in alpha), far above the rounding of sigma and of __expf.  A pixel whose sigma
// exceeds it is skipped by the exact test below as well, so using it as a pre-test (to skip
// the exponential) or for culling (conservative) changes no decision.
__device__ __forceinline__ float sigma_cut(float o) { return __logf(255.f * o) + 1e-3f; }

// Minimum of sigma over the box of pixel centres [bx0, bx1] x [by0, by1] (absolute pixel
// coordinates).  sigma is convex, so the minimum is 0 when the mean lies inside the box and
// otherwise lies on one of the four edges.
__device__ __forceinline__ float box_min_sigma(float bx0, float by0, float bx1, float by1, float u,
                                               float v, float A, float B, float C) {
  const float lx = bx0 - u, hx = bx1 - u;
  const float ly = by0 - v, hy = by1 - v;
  if (lx <= 0.f && hx >= 0.f && ly <= 0.f && hy >= 0.f) return 0.f;
  return fminf(fminf(edge_min_sigma(lx, ly, hy, A, B, C), edge_min_sigma(hx, ly, hy, A, B, C)),
               fminf(edge_min_sigma(ly, lx, hx, C, B, A), edge_min_sigma(hy, lx, hx, C, B, A)));
}

// Conservative per-tile test: true when no pixel centre of the 16x16 tile with origin
// (x0, y0) can reach alpha >= 1/255 for this Gaussian, so the tile can skip it without
// changing any output.
__device__ __forceinline__ bool tile_culled(float x0, float y0, float u, float v, float A, float B,
                                            float C, float o) {
  return box_min_sigma(x0 + 0.5f, y0 + 0.5f, x0 + 15.5f, y0 + 15.5f, u, v, A, B, C) > sigma_cut(o);
}

// Pixel of thread slot t inside a block 16 pixels wide: each warp owns an 8 x 4 strip
// (warps two to a row), more compact than a 16 x 2 row pair, so fewer Gaussians reach a
// strip's box and the per-strip culling drops more (Gaussian, strip) pairs.
constexpr int kStripW = 8, kStripH = 4;
__device__ __forceinline__ int strip_px(int t) { return ((t >> 5) & 1) * kStripW + (t & 7); }
__device__ __forceinline__ int strip_py(int t) { return (t >> 6) * kStripH + ((t & 31) >> 3); }

// Ordered compaction of one flag per thread over a block of NW warps.  Returns the
// position of a kept item (-1 otherwise) and the number kept.  Contains one barrier;
// s_wc (NW ints) must not be reused before the next barrier.
template <int NW = 8>
__device__ __forceinline__ int block_compact_index(bool keep, int* s_wc, int* total) {
  const unsigned b = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_wc[w] = __popc(b);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const int c = s_wc[k];
    off += k < w ? c : 0;
    tot += c;
  }
  *total = tot;
  return keep ? off + __popc(b & ((1u << lane) - 1u)) : -1;
}

}  // namespace gs
