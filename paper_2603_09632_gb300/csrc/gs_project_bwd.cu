// a5: backward of the projection (X-GS App. A: Sigma = R S S^T R^T, Sigma' = J W Sigma
// W^T J^T; SH colour), one thread per Gaussian, and the camera-pose gradient for
// tracking (Eq. 2, App. B).  The pose is perturbed on the left, T <- Exp(xi) T with
// xi = (rho, phi): d p_cam = rho + phi x p_cam, d(W Sigma W^T) = [phi]x Sc - Sc [phi]x,
// and the camera centre moves by -W^T rho.  Per-Gaussian pose terms are reduced per
// block and then by one block in a fixed order (deterministic).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kPB = 128;

constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.54627421529603959f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.8906114426405538f;
constexpr float kC3c = 0.45704579946446572f;
constexpr float kC3d = 0.37317633259011546f;
constexpr float kC3e = 1.4453057213202769f;

// Real SH basis Y[k] and its gradient dY[k] w.r.t. the unit direction (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y, float3* dY) {
  Y[0] = kC0;
  dY[0] = make_float3(0.f, 0.f, 0.f);
  if (DEG < 1) return;
  Y[1] = kC1 * y; dY[1] = make_float3(0.f, kC1, 0.f);
  Y[2] = kC1 * z; dY[2] = make_float3(0.f, 0.f, kC1);
  Y[3] = kC1 * x; dY[3] = make_float3(kC1, 0.f, 0.f);
  if (DEG < 2) return;
  Y[4] = kC2a * x * y; dY[4] = make_float3(kC2a * y, kC2a * x, 0.f);
  Y[5] = kC2a * y * z; dY[5] = make_float3(0.f, kC2a * z, kC2a * y);
  Y[6] = kC2b * (2.f * z * z - x * x - y * y);
  dY[6] = make_float3(-2.f * kC2b * x, -2.f * kC2b * y, 4.f * kC2b * z);
  Y[7] = kC2a * x * z; dY[7] = make_float3(kC2a * z, 0.f, kC2a * x);
  Y[8] = kC2c * (x * x - y * y); dY[8] = make_float3(2.f * kC2c * x, -2.f * kC2c * y, 0.f);
  if (DEG < 3) return;
  Y[9] = kC3a * y * (3.f * x * x - y * y);
  dY[9] = make_float3(6.f * kC3a * x * y, kC3a * (3.f * x * x - 3.f * y * y), 0.f);
  Y[10] = kC3b * x * y * z; dY[10] = make_float3(kC3b * y * z, kC3b * x * z, kC3b * x * y);
  Y[11] = kC3c * y * (4.f * z * z - x * x - y * y);
  dY[11] = make_float3(-2.f * kC3c * x * y, kC3c * (4.f * z * z - x * x - 3.f * y * y), 8.f * kC3c * y * z);
  Y[12] = kC3d * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
  dY[12] = make_float3(-6.f * kC3d * x * z, -6.f * kC3d * y * z, kC3d * (6.f * z * z - 3.f * x * x - 3.f * y * y));
  Y[13] = kC3c * x * (4.f * z * z - x * x - y * y);
  dY[13] = make_float3(kC3c * (4.f * z * z - 3.f * x * x - y * y), -2.f * kC3c * x * y, 8.f * kC3c * x * z);
  Y[14] = kC3e * z * (x * x - y * y);
  dY[14] = make_float3(2.f * kC3e * x * z, -2.f * kC3e * y * z, kC3e * (x * x - y * y));
  Y[15] = kC3a * x * (x * x - 3.f * y * y);
  dY[15] = make_float3(kC3a * (3.f * x * x - 3.f * y * y), -6.f * kC3a * x * y, 0.f);
}

// Rows of a block's outputs staged in shared memory with an odd row stride P (no bank
// conflicts when each thread stores its own row), then written to the row-major global
// array (NF floats per row) with coalesced 16-byte stores when the destination allows.
template <int NF>
struct RowStage {
  static constexpr int P = NF | 1;
  float v[kPB * P];
  __device__ __forceinline__ float* row(int r) { return v + r * P; }
  __device__ __forceinline__ float at(int e) const { return v[(e / NF) * P + e % NF]; }
  __device__ __forceinline__ void write(float* __restrict__ dst, int64_t row0, int rows) const {
    float* base = dst + row0 * NF;
    const int total = rows * NF;
    int e0 = 0;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) == 0) {
      const int nv = total >> 2;
      for (int q = threadIdx.x; q < nv; q += kPB)
        reinterpret_cast<float4*>(base)[q] = make_float4(at(4 * q), at(4 * q + 1), at(4 * q + 2), at(4 * q + 3));
      e0 = nv << 2;
    }
    for (int e = e0 + threadIdx.x; e < total; e += kPB) base[e] = at(e);
  }
};

template <int DEG>
__global__ void __launch_bounds__(kPB)
k_project_bwd(int64_t n, CamDev cam, const float* __restrict__ means,
              const float* __restrict__ scales, const float* __restrict__ quats,
              const float* __restrict__ sh, const GaussRec* __restrict__ rec,
              const uint32_t* __restrict__ ntiles, const float* __restrict__ g2d,
              float* __restrict__ g_means, float* __restrict__ g_scales,
              float* __restrict__ g_quats, float* __restrict__ g_opac, float* __restrict__ g_sh,
              float* __restrict__ pose_partials) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const int64_t row0 = (int64_t)blockIdx.x * kPB;
  const int64_t i = row0 + threadIdx.x;
  const int rows = (int)min64(kPB, n - row0);
  // SH gradient rows (3K floats per Gaussian, K > 1) are written coalesced by the whole
  // block through shared memory; the short rows are stored directly
  __shared__ RowStage<K == 1 ? 1 : K * 3> s_gsh;
  float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < n) {
    const bool valid = ntiles[i] > 0;
    float gm[3] = {0.f, 0.f, 0.f}, gs3[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    float gshv[K * 3];
#pragma unroll
    for (int k = 0; k < K * 3; ++k) gshv[k] = 0.f;
    float gop = 0.f;
    if (valid) {
      const float4* G2 = reinterpret_cast<const float4*>(g2d + i * kG2D);
      const float4 ga = G2[0], gb = G2[1], gc = G2[2];
      const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb.x;
      gop = gb.y;
      const float grgb[3] = {gb.z, gb.w, gc.x};
      const float gz_depth = gc.y;
      const float* R = cam.R;
      const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
      const float x = R[0] * mx + R[1] * my + R[2] * mz + cam.t[0];
      const float y = R[3] * mx + R[4] * my + R[5] * mz + cam.t[1];
      const float z = R[6] * mx + R[7] * my + R[8] * mz + cam.t[2];
      const float4 qv = *reinterpret_cast<const float4*>(quats + 4 * i);
      const float ql = sqrtf(qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w);
      const float w = qv.x / ql, qx = qv.y / ql, qy = qv.z / ql, qz = qv.w / ql;
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
      const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
      float M[9], Sig[9], A[9], Sc[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r * 3 + c] = Rq[r * 3 + c] * s[c];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          Sig[r * 3 + c] = M[r * 3] * M[c * 3] + M[r * 3 + 1] * M[c * 3 + 1] + M[r * 3 + 2] * M[c * 3 + 2];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          A[r * 3 + c] = R[r * 3] * Sig[c] + R[r * 3 + 1] * Sig[3 + c] + R[r * 3 + 2] * Sig[6 + c];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          Sc[r * 3 + c] = A[r * 3] * R[c * 3] + A[r * 3 + 1] * R[c * 3 + 1] + A[r * 3 + 2] * R[c * 3 + 2];
      const float limx = 1.3f * (0.5f * (float)cam.W) / cam.fx;
      const float limy = 1.3f * (0.5f * (float)cam.H) / cam.fy;
      const float iz = 1.f / z;
      const float tx = x * iz, ty = y * iz;
      const bool clx = !(tx > -limx && tx < limx), cly = !(ty > -limy && ty < limy);
      const float txc = fminf(limx, fmaxf(-limx, tx)), tyc = fminf(limy, fmaxf(-limy, ty));
      const float J00 = cam.fx * iz, J02 = -cam.fx * txc * iz;
      const float J11 = cam.fy * iz, J12 = -cam.fy * tyc * iz;
      // conic Q (as rendered) and dL/dcov = -Q Gq Q
      const float4 r0 = rec[i].r0;
      const float4 r1 = rec[i].r1;
      const float Qa = r0.z, Qb = r0.w, Qc = r1.x;
      const float Ga = gA, Gb = 0.5f * gB, Gc = gC;
      const float X00 = Qa * Ga + Qb * Gb, X01 = Qa * Gb + Qb * Gc;
      const float X10 = Qb * Ga + Qc * Gb, X11 = Qb * Gb + Qc * Gc;
      const float C00 = -(X00 * Qa + X01 * Qb);
      const float C01 = -(X00 * Qb + X01 * Qc);
      const float C11 = -(X10 * Qb + X11 * Qc);
      // cov = J Sc J^T + 0.3 I ; J rows: (J00, 0, J02), (0, J11, J12)
      const float Jm[6] = {J00, 0.f, J02, 0.f, J11, J12};
      const float Gc2[4] = {C00, C01, C01, C11};
      float GSc[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) acc += Jm[r * 3 + a] * Gc2[r * 2 + q] * Jm[q * 3 + b];
          GSc[a * 3 + b] = acc;
        }
      float GJ[6];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc += Gc2[r * 2 + q] * Jm[q * 3 + c] * Sc[c * 3 + b];
          GJ[r * 3 + b] = 2.f * acc;
        }
      float gp[3];
      const float iz2 = iz * iz;
      gp[0] = gu * cam.fx * iz;
      gp[1] = gv * cam.fy * iz;
      gp[2] = -gu * cam.fx * x * iz2 - gv * cam.fy * y * iz2 + gz_depth;
      gp[2] += -GJ[0] * cam.fx * iz2 - GJ[4] * cam.fy * iz2;
      gp[2] += GJ[2] * cam.fx * txc * iz2 + GJ[5] * cam.fy * tyc * iz2;
      if (!clx) {
        const float gt = -GJ[2] * cam.fx * iz;
        gp[0] += gt * iz;
        gp[2] += -gt * x * iz2;
      }
      if (!cly) {
        const float gt = -GJ[5] * cam.fy * iz;
        gp[1] += gt * iz;
        gp[2] += -gt * y * iz2;
      }
      // dL/dSigma = W^T GSc W ; dL/dM = 2 GSig M
      float T1[9], GSig[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          T1[a * 3 + b] = R[a] * GSc[b] + R[3 + a] * GSc[3 + b] + R[6 + a] * GSc[6 + b];   // W^T GSc
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          GSig[a * 3 + b] = T1[a * 3] * R[b] + T1[a * 3 + 1] * R[3 + b] + T1[a * 3 + 2] * R[6 + b];
      float GR[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float gmab = 2.f * (GSig[a * 3] * M[b] + GSig[a * 3 + 1] * M[3 + b] + GSig[a * 3 + 2] * M[6 + b]);
          GR[a * 3 + b] = gmab * s[b];
          gs3[b] += gmab * Rq[a * 3 + b];
        }
      float gn[4];
      gn[0] = 2.f * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
      gn[1] = 2.f * (qy * GR[1] + qz * GR[2] + qy * GR[3] - 2.f * qx * GR[4] - w * GR[5] +
                     qz * GR[6] + w * GR[7] - 2.f * qx * GR[8]);
      gn[2] = 2.f * (-2.f * qy * GR[0] + qx * GR[1] + w * GR[2] + qx * GR[3] + qz * GR[5] -
                     w * GR[6] + qz * GR[7] - 2.f * qy * GR[8]);
      gn[3] = 2.f * (-2.f * qz * GR[0] - w * GR[1] + qx * GR[2] + w * GR[3] - 2.f * qz * GR[4] +
                     qy * GR[5] + qx * GR[6] + qy * GR[7]);
      const float qn[4] = {w, qx, qy, qz};
      const float dotn = gn[0] * w + gn[1] * qx + gn[2] * qy + gn[3] * qz;
#pragma unroll
      for (int c = 0; c < 4; ++c) gq[c] = (gn[c] - qn[c] * dotn) / ql;
      // SH colour
      float cp[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) cp[k] = -(R[k] * cam.t[0] + R[3 + k] * cam.t[1] + R[6 + k] * cam.t[2]);
      const float d0 = mx - cp[0], d1 = my - cp[1], d2 = mz - cp[2];
      const float dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      const float dx = d0 / dl, dy = d1 / dl, dz = d2 / dl;
      float Y[K];
      float3 dY[K];
      sh_eval<DEG>(dx, dy, dz, Y, dY);
      const float* shi = sh + i * (K * 3);
      float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float col = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) col += shi[k * 3 + ch] * Y[k];
        if (col + 0.5f <= 0.f) continue;   // colour clamped at 0
        const float gcol = grgb[ch];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          gshv[k * 3 + ch] = gcol * Y[k];
          const float cs = gcol * shi[k * 3 + ch];
          gdir[0] += cs * dY[k].x;
          gdir[1] += cs * dY[k].y;
          gdir[2] += cs * dY[k].z;
        }
      }
      const float dd = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
      const float gdv[3] = {(gdir[0] - dx * dd) / dl, (gdir[1] - dy * dd) / dl, (gdir[2] - dz * dd) / dl};
#pragma unroll
      for (int c = 0; c < 3; ++c) gm[c] = R[c] * gp[0] + R[3 + c] * gp[1] + R[6 + c] * gp[2] + gdv[c];
      // pose twist
#pragma unroll
      for (int c = 0; c < 3; ++c) pose[c] = gp[c] + (R[c * 3] * gdv[0] + R[c * 3 + 1] * gdv[1] + R[c * 3 + 2] * gdv[2]);
      float Am[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < 3; ++r) acc += Sc[a * 3 + r] * GSc[r * 3 + b] - GSc[a * 3 + r] * Sc[r * 3 + b];
          Am[a * 3 + b] = acc;
        }
      pose[3] = (y * gp[2] - z * gp[1]) + (Am[5] - Am[7]);
      pose[4] = (z * gp[0] - x * gp[2]) + (Am[6] - Am[2]);
      pose[5] = (x * gp[1] - y * gp[0]) + (Am[1] - Am[3]);
    }
    if (g_means) { g_means[3 * i] = gm[0]; g_means[3 * i + 1] = gm[1]; g_means[3 * i + 2] = gm[2]; }
    if (g_scales) { g_scales[3 * i] = gs3[0]; g_scales[3 * i + 1] = gs3[1]; g_scales[3 * i + 2] = gs3[2]; }
    if (g_quats)
      *reinterpret_cast<float4*>(g_quats + 4 * i) = make_float4(gq[0], gq[1], gq[2], gq[3]);
    if (g_opac) g_opac[i] = gop;
    if (g_sh) {
      if constexpr (K == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) g_sh[i * 3 + k] = gshv[k];
      } else {
        float* rh = s_gsh.row(threadIdx.x);
#pragma unroll
        for (int k = 0; k < K * 3; ++k) rh[k] = gshv[k];
      }
    }
  }
  if constexpr (K > 1) {
    if (g_sh) {   // uniform
      __syncthreads();
      s_gsh.write(g_sh, row0, rows);
    }
  }
  // block reduction of the pose terms
  __shared__ float s_p[kPB / 32][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float v = pose[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_p[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = 0.f;
    for (int wi = 0; wi < kPB / 32; ++wi) v += s_p[wi][threadIdx.x];
    pose_partials[(int64_t)blockIdx.x * 8 + threadIdx.x] = v;
  }
}

// Sum of the per-block pose partials (stride 8 floats, 6 used) in a fixed order: thread t
// takes blocks t, t + kPR, ... with two 16-byte loads each, then warp and block reductions.
constexpr int kPR = 512;
__global__ void __launch_bounds__(kPR)
k_pose_reduce(const float* __restrict__ partials, int nblocks, float* __restrict__ g_pose6) {
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float4* p4 = reinterpret_cast<const float4*>(partials);
#pragma unroll 4
  for (int b = threadIdx.x; b < nblocks; b += kPR) {
    const float4 u = p4[2 * b], v = p4[2 * b + 1];
    acc[0] += u.x;
    acc[1] += u.y;
    acc[2] += u.z;
    acc[3] += u.w;
    acc[4] += v.x;
    acc[5] += v.y;
  }
  __shared__ float s[kPR / 32][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float x = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][c] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float x = 0.f;
    for (int w = 0; w < kPR / 32; ++w) x += s[w][threadIdx.x];
    g_pose6[threadIdx.x] = x;
  }
}

__global__ void k_l1_grad(const float* __restrict__ pred, const float* __restrict__ target,
                          int64_t n, float scale, float* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float d = pred[i] - target[i];
    grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  }
}

}  // namespace

int project_bwd_blocks(int64_t n) { return (int)ceil_div(max64(n, 1), kPB); }

void launch_project_bwd(const gs_scene& sc, const CamDev& cam, const GaussRec* rec,
                        const uint32_t* ntiles, const float* g2d, float* g_means, float* g_scales,
                        float* g_quats, float* g_opac, float* g_sh, float* pose_partials,
                        float* g_pose6, cudaStream_t st) {
  const int nb = project_bwd_blocks(sc.n);
  if (sc.n > 0) {
#define GS_PB(d)                                                                                   \
  k_project_bwd<d><<<nb, kPB, 0, st>>>(sc.n, cam, sc.means, sc.scales, sc.quats, sc.sh, rec, ntiles, \
                                       g2d, g_means, g_scales, g_quats, g_opac, g_sh, pose_partials)
    switch (sc.sh_degree) {
      case 0: GS_PB(0); break;
      case 1: GS_PB(1); break;
      case 2: GS_PB(2); break;
      default: GS_PB(3); break;
    }
#undef GS_PB
    note_launch();
  }
  if (g_pose6) {
    if (sc.n > 0) {
      k_pose_reduce<<<1, kPR, 0, st>>>(pose_partials, nb, g_pose6);
      note_launch();
    } else {
      cudaMemsetAsync(g_pose6, 0, 6 * sizeof(float), st);
    }
  }
}

void launch_l1_grad(const float* pred, const float* target, int64_t n, float scale, float* grad,
                    cudaStream_t st) {
  if (n <= 0) return;
  k_l1_grad<<<(int)ceil_div(n, 256), 256, 0, st>>>(pred, target, n, scale, grad);
  note_launch();
}

}  // namespace gs
