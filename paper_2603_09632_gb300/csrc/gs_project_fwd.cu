// a1: EWA projection + SH colour, one thread per Gaussian (X-GS App. A:
// Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T; colour from real SH along the
// view direction).
//
// This translation unit is compiled with -fmad=false: every key-affecting value
// (camera-space depth, 2D mean, the 2D covariance feeding the 3-sigma radius and the
// tile rectangle) is computed with separately rounded IEEE operations in one fixed
// order, so that tile keys and sorted lists are reproducible bit for bit by any
// implementation that follows the same order.  The order is written out below.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kProjThreads = 128;

// Real SH basis constants (orthonormal, no Condon-Shortley phase).
constexpr float kC0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kC1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kC2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kC3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kC3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kC3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kC3d = 0.37317633259011546f;  // sqrt(7 / pi) / 4
constexpr float kC3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

// Copy rows [row0, row0+rows) of a row-major float array with nf floats per row into
// shared memory, with 16-byte loads when the source is 16-byte aligned.
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, int64_t row0, int rows,
                                           int nf, float* __restrict__ dst) {
  const float* base = src + row0 * nf;
  const int total = rows * nf;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) == 0) {
    const int nv = total >> 2;
    const float4* b4 = reinterpret_cast<const float4*>(base);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) d4[i] = __ldg(b4 + i);
    for (int i = (nv << 2) + threadIdx.x; i < total; i += blockDim.x) dst[i] = __ldg(base + i);
  } else {
    for (int i = threadIdx.x; i < total; i += blockDim.x) dst[i] = __ldg(base + i);
  }
}

__device__ __forceinline__ float clamp_tile(float f, int hi) {
  return fminf(fmaxf(f, 0.f), (float)hi);
}

// At most 40 registers: 12 resident CTAs per SM, so that a few hundred thousand Gaussians
// are projected in one wave (most of them leave at the frustum test).
template <int DEG>
__global__ void __launch_bounds__(kProjThreads, 12)
k_project(int64_t n, CamDev cam, const float* __restrict__ means, const float* __restrict__ scales,
          const float* __restrict__ quats, const float* __restrict__ opac,
          const float* __restrict__ sh, GaussRec* __restrict__ rec,
          uint32_t* __restrict__ depth_key, uint32_t* __restrict__ ntiles,
          uint2* __restrict__ rect, uint32_t* __restrict__ counters,
          uint32_t* __restrict__ tile_count) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ __align__(16) float s_mu[kProjThreads * 3];
  __shared__ __align__(16) float s_sc[kProjThreads * 3];
  __shared__ __align__(16) float s_q[kProjThreads * 4];
  // SH degree 0 is staged with the geometry; higher degrees (up to 192 B per Gaussian) are
  // read from global memory by the visible Gaussians only
  __shared__ __align__(16) float s_sh[K == 1 ? kProjThreads * 3 : 1];
  const int64_t row0 = (int64_t)blockIdx.x * kProjThreads;
  const int rows = (int)min64(kProjThreads, n - row0);
  stage_rows(means, row0, rows, 3, s_mu);
  stage_rows(scales, row0, rows, 3, s_sc);
  stage_rows(quats, row0, rows, 4, s_q);
  if (K == 1) stage_rows(sh, row0, rows, 3, s_sh);
  __syncthreads();
  const int l = threadIdx.x;
  uint32_t cnt_v = 0, cnt_i = 0;
  uint2 rc_l = make_uint2(0u, 0u);   // this lane's rectangle and tile count for the binning
  if (l < rows) {
    const int64_t i = row0 + l;

    const float* R = cam.R;
    const float mx = s_mu[3 * l], my = s_mu[3 * l + 1], mz = s_mu[3 * l + 2];
    // p = W mu + t
    const float x = ((R[0] * mx + R[1] * my) + R[2] * mz) + cam.t[0];
    const float y = ((R[3] * mx + R[4] * my) + R[5] * mz) + cam.t[1];
    const float z = ((R[6] * mx + R[7] * my) + R[8] * mz) + cam.t[2];

    uint32_t nt = 0;
    uint2 rc = make_uint2(0, 0);
    GaussRec g;
    g.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    g.r1 = g.r0;
    g.r2 = g.r0;
    bool valid = z > cam.near_z;
    float a = 0.f, b = 0.f, c = 0.f, det = 0.f, u = 0.f, v = 0.f;
    if (valid) {
      // unit quaternion (w, x, y, z) -> rotation
      const float q0 = s_q[4 * l], q1 = s_q[4 * l + 1], q2 = s_q[4 * l + 2], q3 = s_q[4 * l + 3];
      const float ql = sqrtf(((q0 * q0 + q1 * q1) + q2 * q2) + q3 * q3);
      const float w = q0 / ql, qx = q1 / ql, qy = q2 / ql, qz = q3 / ql;
      float Rq[9];
      Rq[0] = 1.f - 2.f * (qy * qy + qz * qz);
      Rq[1] = 2.f * (qx * qy - w * qz);
      Rq[2] = 2.f * (qx * qz + w * qy);
      Rq[3] = 2.f * (qx * qy + w * qz);
      Rq[4] = 1.f - 2.f * (qx * qx + qz * qz);
      Rq[5] = 2.f * (qy * qz - w * qx);
      Rq[6] = 2.f * (qx * qz - w * qy);
      Rq[7] = 2.f * (qy * qz + w * qx);
      Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
      const float s0 = s_sc[3 * l], s1 = s_sc[3 * l + 1], s2 = s_sc[3 * l + 2];
      float M[9];
  #pragma unroll
      for (int r = 0; r < 3; ++r) {
        M[r * 3 + 0] = Rq[r * 3 + 0] * s0;
        M[r * 3 + 1] = Rq[r * 3 + 1] * s1;
        M[r * 3 + 2] = Rq[r * 3 + 2] * s2;
      }
      // Sigma = M M^T (upper triangle, mirrored)
      float Sig[9];
  #pragma unroll
      for (int r = 0; r < 3; ++r)
  #pragma unroll
        for (int s = r; s < 3; ++s) {
          const float e = (M[r * 3] * M[s * 3] + M[r * 3 + 1] * M[s * 3 + 1]) + M[r * 3 + 2] * M[s * 3 + 2];
          Sig[r * 3 + s] = e;
          Sig[s * 3 + r] = e;
        }
      // Sc = W Sigma W^T (A = W Sigma full, then upper triangle of A W^T)
      float A[9];
  #pragma unroll
      for (int r = 0; r < 3; ++r)
  #pragma unroll
        for (int s = 0; s < 3; ++s)
          A[r * 3 + s] = (R[r * 3] * Sig[s] + R[r * 3 + 1] * Sig[3 + s]) + R[r * 3 + 2] * Sig[6 + s];
      float Sc[9];
  #pragma unroll
      for (int r = 0; r < 3; ++r)
  #pragma unroll
        for (int s = r; s < 3; ++s) {
          const float e = (A[r * 3] * R[s * 3] + A[r * 3 + 1] * R[s * 3 + 1]) + A[r * 3 + 2] * R[s * 3 + 2];
          Sc[r * 3 + s] = e;
          Sc[s * 3 + r] = e;
        }
      // J with the 1.3 x half-FOV guard band
      const float tanx = (0.5f * (float)cam.W) / cam.fx, tany = (0.5f * (float)cam.H) / cam.fy;
      const float limx = 1.3f * tanx, limy = 1.3f * tany;
      const float tx = x / z, ty = y / z;
      const float txc = fminf(limx, fmaxf(-limx, tx)), tyc = fminf(limy, fmaxf(-limy, ty));
      const float j00 = cam.fx / z, j02 = -((cam.fx * txc) / z);
      const float j11 = cam.fy / z, j12 = -((cam.fy * tyc) / z);
      const float T00 = j00 * Sc[0] + j02 * Sc[2];
      const float T01 = j00 * Sc[1] + j02 * Sc[5];
      const float T02 = j00 * Sc[2] + j02 * Sc[8];
      const float T11 = j11 * Sc[4] + j12 * Sc[5];
      const float T12 = j11 * Sc[5] + j12 * Sc[8];
      a = (T00 * j00 + T02 * j02) + 0.3f;
      b = T01 * j11 + T02 * j12;
      c = (T11 * j11 + T12 * j12) + 0.3f;
      det = a * c - b * b;
      valid = det > 0.f;
      if (valid) {
        const float mid = 0.5f * (a + c);
        const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        const float r = ceilf(3.f * sqrtf(lam));
        u = cam.fx * tx + cam.cx;
        v = cam.fy * ty + cam.cy;
        const int x0 = (int)clamp_tile(floorf((u - r) / 16.f), cam.TX);
        const int x1 = (int)clamp_tile(floorf((u + r) / 16.f) + 1.f, cam.TX);
        const int y0 = (int)clamp_tile(floorf((v - r) / 16.f), cam.TY);
        const int y1 = (int)clamp_tile(floorf((v + r) / 16.f) + 1.f, cam.TY);
        valid = x1 > x0 && y1 > y0;
        if (valid) {
          nt = (uint32_t)((x1 - x0) * (y1 - y0));
          rc = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
        }

      }
    }
    if (valid) {
      // colour: real SH along dir = normalize(mu - camera centre), camera centre = -W^T t
      float cp[3];
  #pragma unroll
      for (int k = 0; k < 3; ++k)
        cp[k] = -((R[k] * cam.t[0] + R[3 + k] * cam.t[1]) + R[6 + k] * cam.t[2]);
      const float d0 = mx - cp[0], d1 = my - cp[1], d2 = mz - cp[2];
      const float dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      const float dx = d0 / dl, dy = d1 / dl, dz = d2 / dl;
      float Y[K];
      Y[0] = kC0;
      if (DEG >= 1) {
        Y[1] = kC1 * dy;
        Y[2] = kC1 * dz;
        Y[3] = kC1 * dx;
      }
      if (DEG >= 2) {
        Y[4] = kC2a * dx * dy;
        Y[5] = kC2a * dy * dz;
        Y[6] = kC2b * (2.f * dz * dz - dx * dx - dy * dy);
        Y[7] = kC2a * dx * dz;
        Y[8] = kC2c * (dx * dx - dy * dy);
      }
      if (DEG >= 3) {
        Y[9] = kC3a * dy * (3.f * dx * dx - dy * dy);
        Y[10] = kC3b * dx * dy * dz;
        Y[11] = kC3c * dy * (4.f * dz * dz - dx * dx - dy * dy);
        Y[12] = kC3d * dz * (2.f * dz * dz - 3.f * dx * dx - 3.f * dy * dy);
        Y[13] = kC3c * dx * (4.f * dz * dz - dx * dx - dy * dy);
        Y[14] = kC3e * dz * (dx * dx - dy * dy);
        Y[15] = kC3a * dx * (dx * dx - 3.f * dy * dy);
      }
      const float* shl = K == 1 ? s_sh + l * 3 : sh + i * (K * 3);
      float col[3];
  #pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
  #pragma unroll
        for (int k = 0; k < K; ++k) acc += (K == 1 ? shl[k * 3 + ch] : __ldg(shl + k * 3 + ch)) * Y[k];
        acc += 0.5f;
        col[ch] = acc > 0.f ? acc : 0.f;
      }
      g.r0 = make_float4(u, v, c / det, -b / det);
      g.r1 = make_float4(a / det, __ldg(opac + i), z, 0.f);
      g.r2 = make_float4(col[0], col[1], col[2], 0.f);
    }
    if (valid) {   // records and keys are read only for Gaussians with tiles
      rec[i] = g;
      depth_key[i] = __float_as_uint(z);
    }
    ntiles[i] = nt;
    rect[i] = rc;
    cnt_v = valid ? 1u : 0u;
    cnt_i = nt;
    rc_l = rc;
  }
  // per-tile instance counts for the binning (the count step of the tile buckets): per-row
  // differences on large frames, per-tile counts otherwise (uniform over the launch)
  if (tile_count) {
    if (count_tile_rows(cam.TX * cam.TY))
      warp_count_rows(cnt_i, rc_l, cam.TX, tile_count);
    else
      warp_count_tiles(cnt_i, rc_l, cam.TX, cam.TX * cam.TY, tile_count);
  }
  // V and I for the workspace counters: warp sums, then one atomic per block
  __shared__ uint32_t s_cnt[2];
  if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0u;
  __syncthreads();
  cnt_v = __reduce_add_sync(0xffffffffu, cnt_v);
  cnt_i = __reduce_add_sync(0xffffffffu, cnt_i);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_cnt[0], cnt_v);
    atomicAdd(&s_cnt[1], cnt_i);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(&counters[kCntVisible], s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&counters[kCntInst], s_cnt[1]);
  }
}

}  // namespace

void launch_project(const gs_scene& sc, const CamDev& cam, GaussRec* rec, uint32_t* depth_key,
                    uint32_t* ntiles, uint2* rect, uint32_t* counters, uint32_t* tile_count,
                    cudaStream_t st) {
  if (sc.n <= 0) return;
  const int grid = (int)ceil_div(sc.n, kProjThreads);
  switch (sc.sh_degree) {
    case 0: k_project<0><<<grid, kProjThreads, 0, st>>>(sc.n, cam, sc.means, sc.scales, sc.quats, sc.opacities, sc.sh, rec, depth_key, ntiles, rect, counters, tile_count); break;
    case 1: k_project<1><<<grid, kProjThreads, 0, st>>>(sc.n, cam, sc.means, sc.scales, sc.quats, sc.opacities, sc.sh, rec, depth_key, ntiles, rect, counters, tile_count); break;
    case 2: k_project<2><<<grid, kProjThreads, 0, st>>>(sc.n, cam, sc.means, sc.scales, sc.quats, sc.opacities, sc.sh, rec, depth_key, ntiles, rect, counters, tile_count); break;
    default: k_project<3><<<grid, kProjThreads, 0, st>>>(sc.n, cam, sc.means, sc.scales, sc.quats, sc.opacities, sc.sh, rec, depth_key, ntiles, rect, counters, tile_count); break;
  }
  note_launch();
}

}  // namespace gs
