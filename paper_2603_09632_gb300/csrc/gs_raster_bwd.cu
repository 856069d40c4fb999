// a4: backward of the tile rasterizer (X-GS App. B: the rasterizer is differentiable;
// Eq. 2 tracking and Eq. 3 mapping need dL/dTheta and dL/dT).
//
// Per pixel, with w_i = a_i T_i and T_i = prod_{j<i}(1 - a_j):
//   dL/dc_i = w_i g_C,  dL/dd_i = w_i g_D,  dL/df_i = w_i g_F
//   dL/da_i = T_i (g.x_i - s_i) + g_A T_final / (1 - a_i),   x_i = (c_i, d_i, f_i)
//   s_{i-1} = a_i (g.x_i) + (1 - a_i) s_i   (scalar running sum behind i, s_last = 0)
// and a_i = o_i exp(-sigma_i) gives dL/do_i and dL/dsigma_i, from which the conic and
// 2D-mean gradients follow.
//
// One 256-thread CTA per tile walks the tile's list backwards from the longest pixel
// prefix (max n_contrib), recovering T_i = T_{i+1} / (1 - a_i) from T_final.  The list is
// taken in chunks of 256 entries; each chunk is gathered once, entries that no pixel of
// the tile can blend are dropped (conservative test, outputs unchanged) and the rest are
// compacted into shared memory.  The compacted chunk is processed in batches of B
// Gaussians.  Phase 1 (one thread per pixel, branch-free over the batch's live entries, with
// g.x_i formed ahead of the blend decision so that it overlaps the opacity evaluation)
// writes w and dL/do of each (pixel, Gaussian) pair to shared memory (dL/dsigma = -o dL/do where the alpha cap does not hold, so it is
// not stored).  Phase 2 reduces over the 256 pixels of the
// tile: the feature gradient is the contraction W^T g_F with 4x4 register blocks (pixel
// parts summed through per-warp partials in shared memory, in a fixed order), and
// colour/depth/opacity sums and the pixel moments sum_p dL/dsigma * (1, x, y, xx, xy, yy)
// (from which the conic and mean gradients are formed exactly) are warp reductions.
// The next batch's features are fetched into registers during phase 2.  Two barriers
// per batch.  Each Gaussian receives one 16-byte vector atomic per 4 quantities per tile.
//
// Features-only variant (FO, the semantic phase of Sec. 3.2 where geometry and colour are
// frozen): only dL/df_i = sum_p w_i g_F is needed, so phase 1 keeps just the weights, the
// features themselves are not fetched, and phase 2b and every geometry accumulator are
// skipped.
#include <algorithm>

#include "gs_blend.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kT = 256;        // threads = pixels per tile = entries per chunk
constexpr int kWS = kT + 4;    // row stride of the j-major pair arrays (floats)

template <int DP, bool FO = false>
struct BwdCfg {
  // Gaussians per batch: 8 where a 16-Gaussian batch would leave room for only one
  // resident CTA (64 channels features-only)
  static constexpr int B = (DP >= 64 && FO) ? 8 : 16;
  static constexpr int ES = DP + 4;                     // row stride of s_E (floats)
  static constexpr int JB = B / 4;                      // 4x4 blocks of the contraction
  static constexpr int CB = DP / 4;
  static constexpr int TASKS = JB * CB;
  static constexpr int S = TASKS > 0 ? kT / TASKS : 1;  // pixel split per block
  static constexpr int PP = kT / S;                     // pixels per part
  static constexpr int G = kT / B;                      // threads per Gaussian in phase 2b
  static constexpr int NW = kT / 32;                    // warps
  static constexpr int PW = TASKS > 0 && TASKS < 32 ? 32 / TASKS : 1;   // parts per warp
  static_assert(PW == 1 || PW == 2 || PW == 4, "parts of a warp merged by one or two shuffles");
  static_assert(TASKS == 0 || TASKS % 32 == 0 || 32 % TASKS == 0, "tasks tile the warps");
  static constexpr size_t base_floats =
      (size_t)kT * ES           // s_E: upstream feature gradient per pixel
      + (size_t)(FO ? 1 : 2) * B * kWS   // s_W (and s_GO unless FO), j-major
      + (size_t)(FO ? 0 : 2) * B * DP;  // s_f: batch features, double buffered (not when FO)
  // Feature-gradient sums of a batch: one partial [B][DP] per warp (parts of a warp merged
  // by shuffles) or per part (a part spanning several warps), added in order by the flush:
  // no shared-memory atomics, and a fixed summation order.
  static constexpr int NPART = PW > 1 ? NW : S;
  static constexpr size_t smem_floats = base_floats + (size_t)NPART * B * DP;   // + s_outF
  static constexpr size_t kSM = 228 * 1024, kStatic = 19 * 1024, kReserve = 1024;
  static constexpr int CTAS = 2 * (kStatic + 4 * smem_floats + kReserve) <= kSM ? 2 : 1;   // per SM
};

// Features of one batch: fetched into registers, stored to shared memory later.
template <int DP, bool BF16, int B>
struct FeatBatch {
  static constexpr int VPC = BF16 ? 8 : 4;                 // values per 16-byte chunk
  static constexpr int CPR = DP / VPC > 0 ? DP / VPC : 1;  // chunks per row
  static constexpr int NS = (B * DP + kT - 1) / kT;        // scalar path values per thread
  uint4 v;
  float s[NS > 0 ? NS : 1];

  __device__ __forceinline__ void fetch(const void* __restrict__ feats, int D,
                                        const uint32_t* __restrict__ s_id, int jb0, int bc) {
    const int t = threadIdx.x;
    if (D == DP) {
      v = make_uint4(0u, 0u, 0u, 0u);
      if (t < B * CPR) {
        const int j = t / CPR, part = t - j * CPR;
        if (j < bc) {
          const int64_t row = (int64_t)s_id[jb0 + j] * DP;
          if constexpr (BF16)
            v = __ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(feats) + row) + part);
          else
            v = __ldg(reinterpret_cast<const uint4*>(static_cast<const float*>(feats) + row) + part);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int e = t + k * kT;
        float x = 0.f;
        if (e < B * DP) {
          const int j = e / DP, c = e - j * DP;
          if (j < bc && c < D) {
            const int64_t idx = (int64_t)s_id[jb0 + j] * D + c;
            if constexpr (BF16)
              x = __bfloat162float(static_cast<const __nv_bfloat16*>(feats)[idx]);
            else
              x = __ldg(static_cast<const float*>(feats) + idx);
          }
        }
        s[k] = x;
      }
    }
  }

  __device__ __forceinline__ void store(int D, float* __restrict__ s_f) const {
    const int t = threadIdx.x;
    if (D == DP) {
      if (t < B * CPR) {
        const int j = t / CPR, part = t - j * CPR;
        float* dst = s_f + j * DP + part * VPC;
        if constexpr (BF16) {
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            dst[2 * k] = __uint_as_float(w[k] << 16);
            dst[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
          }
        } else {
          *reinterpret_cast<uint4*>(dst) = v;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int e = t + k * kT;
        if (e < B * DP) s_f[e] = s[k];
      }
    }
  }
};

__device__ __forceinline__ void red_add4(float* dst, float a, float b, float c, float d) {
  atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a, b, c, d));
}

// J: the renders of this launch (one for a plain backward, up to kMaxJobs for a serving
// batch); their tiles are taken from one queue.
template <int DP, bool BF16, bool FO, int NJ>
__global__ void __launch_bounds__(kT, (BwdCfg<DP, FO>::CTAS))
k_raster_bwd(const __grid_constant__ RasterJobs<NJ> J, TileQueue tq) {
  using Cfg = BwdCfg<DP, FO>;
  constexpr int B = Cfg::B;
  __shared__ float4 s_r0[kT], s_r1[kT], s_r2[kT];   // compacted records of the chunk
  __shared__ uint32_t s_id[kT];
  __shared__ int s_orig[kT];                        // list position of each compacted entry
  __shared__ float4 s_E4[kT];                       // (g_r, g_g, g_b, g_depth) per pixel
  __shared__ int s_wc[8];
  __shared__ unsigned s_live[8];                    // per warp strip: batch entries that can reach it
  __shared__ uint32_t s_maxn;
  extern __shared__ __align__(16) float smem[];
  float* s_E = smem;                          // [kT][ES]
  float* s_W = s_E + kT * Cfg::ES;            // [B][kWS]
  float* s_GO = s_W + B * kWS;                // (not allocated when FO)
  float* s_fb = s_W + (FO ? 1 : 2) * B * kWS; // [2][B][DP]
  float* s_outF = s_fb + (FO ? 0 : 2) * B * DP;   // [NPART][B][DP] partial sums

  const int t = threadIdx.x;
  __shared__ int s_tile, s_job;
  // persistent CTA: tiles from the queue, heaviest first
  for (;;) {
    if (t == 0) {
      const uint32_t q = atomicAdd(tq.head, 1u);
      s_tile = -1;
      if (q < J.items()) {
        uint32_t first;
        const int k = J.find(q, &first);
        const uint32_t local = q - first;
        const uint32_t* order = J.job[k].order;
        s_tile = (int)(order ? order[local] : local);
        s_job = k;
      }
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) break;
    const RasterJob& jb = J.job[NJ > 1 ? s_job : 0];
    const CamDev& cam = jb.cam;
    const GaussRec* __restrict__ rec = jb.rec;
    const void* __restrict__ feats = jb.feats;
    const int D = jb.D;
    const uint2* __restrict__ ranges = jb.ranges;
    const uint32_t* __restrict__ inst_id = jb.inst_id;
    const float* __restrict__ T_final = jb.T_final;
    const uint32_t* __restrict__ n_contrib = jb.n_contrib;
    const float *__restrict__ g_rgb = jb.g_rgb, *__restrict__ g_depth = jb.g_depth;
    const float *__restrict__ g_alpha = jb.g_alpha, *__restrict__ g_feat = jb.g_feat;
    float* __restrict__ g2d = jb.g2d;
    float* __restrict__ g_feats = jb.g_feats;
    const int tx0 = (tile % cam.TX) * kTile, ty0 = (tile / cam.TX) * kTile;
    const int px = tx0 + strip_px(t), py = ty0 + strip_py(t);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const int lane = t & 31;
    // pixel-centre boxes of the tile and of this warp's 8 x 4 strip
    const float bx0 = (float)tx0 + 0.5f, by0 = (float)ty0 + 0.5f;
    const float wbx0 = (float)(tx0 + strip_px(t & ~31)) + 0.5f;
    const float wby0 = (float)(ty0 + strip_py(t & ~31)) + 0.5f;
    const int64_t HW = (int64_t)cam.W * cam.H;
    const int64_t p = (int64_t)py * cam.W + px;
    const uint2 rg = ranges[tile];
    const int start = (int)rg.x;

    // upstream gradients of this pixel
    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f, Tf = 1.f;
    int nc = 0;
    float2 gF[DP > 0 ? DP / 2 : 1];   // upstream feature gradient in packed pairs
  #pragma unroll
    for (int c = 0; c < (DP > 0 ? DP / 2 : 1); ++c) gF[c] = make_float2(0.f, 0.f);
    if (inside) {
      if (!FO && g_rgb) {
        gC0 = g_rgb[p];
        gC1 = g_rgb[HW + p];
        gC2 = g_rgb[2 * HW + p];
      }
      if (!FO && g_depth) gD = g_depth[p];
      if (!FO && g_alpha) gA = g_alpha[p];
      Tf = T_final[p];
      nc = (int)n_contrib[p];
      if constexpr (DP > 0) {
  #pragma unroll
        for (int c = 0; c < DP; c += 2)
          gF[c / 2] = make_float2(c < D ? g_feat[c * HW + p] : 0.f, c + 1 < D ? g_feat[(c + 1) * HW + p] : 0.f);
      }
    }
    if constexpr (DP > 0) {
  #pragma unroll
      for (int c = 0; c < DP; c += 4)
        *reinterpret_cast<float4*>(s_E + t * Cfg::ES + c) =
            make_float4(gF[c / 2].x, gF[c / 2].y, gF[c / 2 + 1].x, gF[c / 2 + 1].y);
    }
    s_E4[t] = make_float4(gC0, gC1, gC2, gD);
    if (t == 0) s_maxn = 0;
    __syncthreads();
    if (nc > 0) atomicMax(&s_maxn, (uint32_t)nc);
    const int warp_nc = (int)__reduce_max_sync(0xffffffffu, (unsigned)nc);   // this strip's
    __syncthreads();
    const int maxn = (int)s_maxn;
    if (rg.x + (uint32_t)maxn <= rg.y) {          // always, for consistent inputs

    float T = Tf, s_run = 0.f;
    const float gAT = gA * Tf;

    for (int c1 = maxn; c1 > 0; c1 -= kT) {
      const int c0 = max(0, c1 - kT);
      // ---- gather the chunk [c0, c1) of the list, drop entries the tile cannot blend
      __syncthreads();                          // previous chunk fully consumed
      bool keep = false;
      uint32_t id = 0;
      GaussRec g;
      if (t < c1 - c0) id = inst_id[start + c0 + t];
      if (t < c1 - c0 && id < (uint32_t)cam.n_gauss) {
        g = rec[id];
        g.r1.w = sigma_cut(g.r1.y);
        keep = box_min_sigma(bx0, by0, bx0 + 15.f, by0 + 15.f, g.r0.x, g.r0.y, g.r0.z, g.r0.w,
                             g.r1.x) <= g.r1.w;
      }
      int nk;
      const int pos = block_compact_index(keep, s_wc, &nk);
      if (keep) {
        s_r0[pos] = g.r0;
        s_r1[pos] = g.r1;
        s_r2[pos] = g.r2;
        s_id[pos] = id;
        s_orig[pos] = c0 + t;
      }
      __syncthreads();
      FeatBatch<DP, BF16, B> fb;
      if constexpr (DP > 0 && !FO) {
        fb.fetch(feats, D, s_id, max(0, nk - B), min(B, nk));
        fb.store(D, s_fb);
        __syncthreads();
      }

      // ---- batches of the compacted chunk, last entries first
      for (int jb1 = nk, bi = 0; jb1 > 0; jb1 -= B, ++bi) {
        const int jb0 = max(0, jb1 - B), bc = jb1 - jb0;
        const float* s_f = s_fb + (bi & 1) * B * DP;

        // entries of the batch that can reach this warp's 8 x 4 pixel strip
        bool hit = false;
        if (lane < bc) {
          const float4 q0 = s_r0[jb0 + lane], q1 = s_r1[jb0 + lane];
          hit = box_min_sigma(wbx0, wby0, wbx0 + (float)(kStripW - 1), wby0 + (float)(kStripH - 1),
                              q0.x, q0.y, q0.z, q0.w, q1.x) <= q1.w;
        }
        // ... and that some pixel of the strip still blends (list position below the strip's
        // largest last-contributor count)
        if (lane < bc) hit = hit && s_orig[jb0 + lane] < warp_nc;
        const unsigned live = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) s_live[t >> 5] = live;   // phase 2 skips (Gaussian, strip) pairs not live

        // phase 1: per pixel, reverse over the batch
        for (int j = B - 1; j >= 0; --j) {
          if (!(live >> j & 1u)) continue;   // entries not live for this strip are never read
          float w = 0.f, go = 0.f;
          const float4 r0 = s_r0[jb0 + j];
          const float4 r1 = s_r1[jb0 + j];
          // g.x_i does not depend on the blend decisions below: it is formed on every lane
          // of a live entry, so that it overlaps the opacity evaluation
          float dot = 0.f;
          if constexpr (!FO) {
            const float4 r2 = s_r2[jb0 + j];
            float2 d01 = mul2(make_float2(gC0, gC1), make_float2(r2.x, r2.y));
            float2 d23 = mul2(make_float2(gC2, gD), make_float2(r2.z, r1.z));
            if constexpr (DP > 0) {
              const float4* f4 = reinterpret_cast<const float4*>(s_f + j * DP);
  #pragma unroll
              for (int q = 0; q < DP / 4; ++q) {
                const float4 f = f4[q];
                d01 = fma2(gF[2 * q], make_float2(f.x, f.y), d01);
                d23 = fma2(gF[2 * q + 1], make_float2(f.z, f.w), d23);
              }
            }
            dot = (d01.x + d01.y) + (d23.x + d23.y);
          }
          const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
          // branch-free: every lane evaluates, and the blend decision selects the updates
          // (the same values as the branches would give), so consecutive entries overlap
          const float G = blend_gauss(sigma);
          const float oG = __fmul_rn(r1.y, G);
          const float a = fminf(kAlphaMax, oG);
          const bool ok = (s_orig[jb0 + j] < nc) & (sigma >= 0.f) & (sigma <= r1.w) & (a >= kAlphaMin);
          const float inv = __fdividef(1.f, 1.f - a);
          const float Tn = T * inv;                 // T_i
          if (ok) w = a * Tn;
          if constexpr (!FO) {
            const float galpha = Tn * (dot - s_run) + gAT * inv;
            const float sn = a * dot + (1.f - a) * s_run;
            // dL/do = galpha G; dL/dsigma = -galpha a = -o dL/do (phase 2b scales the
            // moments of dL/do by -o); both zero where the 0.99 cap holds alpha
            if (ok && oG <= kAlphaMax) go = galpha * G;
            if (ok) s_run = sn;
          }
          if (ok) T = Tn;
          s_W[j * kWS + t] = w;
          if constexpr (!FO) s_GO[j * kWS + t] = go;
        }
        __syncthreads();

        // next batch's features: fetch now, store after phase 2
        const bool more = jb0 > 0;
        if constexpr (DP > 0 && !FO) {
          if (more) fb.fetch(feats, D, s_id, max(0, jb0 - B), min(B, jb0));
        }

        // phase 2a: feature gradients, out[j][c] = sum_p W[j][p] g_F[p][c]
        if constexpr (DP > 0) {
          if (g_feats) {
            const int cb = t % Cfg::CB;
            const int jb = (t / Cfg::CB) % Cfg::JB;
            const int part = t / Cfg::TASKS;
            constexpr int PP = Cfg::PP;
            float2 acc[4][2];   // rows a, columns in packed pairs
  #pragma unroll
            for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
            // a part lies in one warp strip or spans whole strips; W holds values only where
            // the Gaussian is live for the strip, so liveness is applied strip by strip
            constexpr int NSP = PP >= 32 ? PP / 32 : 1;   // strips per part
            constexpr int QS = PP >= 32 ? 32 : PP;        // pixels per (part, strip)
            const int p0 = part * PP;
  #pragma unroll
            for (int ws = 0; ws < NSP; ++ws) {
              const int q0 = p0 + ws * QS;
              const unsigned lv = (s_live[q0 >> 5] >> (4 * jb)) & 15u;
  #pragma unroll 4
              for (int q = q0; q < (lv ? q0 + QS : q0); q += 4) {
                float4 wv[4], ev[4];
  #pragma unroll
                for (int a = 0; a < 4; ++a)
                  wv[a] = (lv >> a & 1u) ? *reinterpret_cast<const float4*>(s_W + (4 * jb + a) * kWS + q)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
  #pragma unroll
                for (int b = 0; b < 4; ++b) ev[b] = *reinterpret_cast<const float4*>(s_E + (q + b) * Cfg::ES + 4 * cb);
  #pragma unroll
                for (int a = 0; a < 4; ++a) {
                  const float wa[4] = {wv[a].x, wv[a].y, wv[a].z, wv[a].w};
  #pragma unroll
                  for (int b = 0; b < 4; ++b) {
                    const float2 w2 = splat2(wa[b]);
                    acc[a][0] = fma2(w2, make_float2(ev[b].x, ev[b].y), acc[a][0]);
                    acc[a][1] = fma2(w2, make_float2(ev[b].z, ev[b].w), acc[a][1]);
                  }
                }
              }
            }
            // merge the PW parts of this warp (lanes TASKS apart) by a reduce-scatter: first
            // over the rows a, then (PW = 4) over the columns b; each lane then stores its
            // share of this warp's partial [B][DP] (PW = 1: its task's block of its part's)
            float* dst = s_outF + (Cfg::PW > 1 ? t >> 5 : part) * (B * DP) + 4 * cb;
            if constexpr (Cfg::PW == 1) {
  #pragma unroll
              for (int a = 0; a < 4; ++a)
                *reinterpret_cast<float4*>(dst + (4 * jb + a) * DP) =
                    make_float4(acc[a][0].x, acc[a][0].y, acc[a][1].x, acc[a][1].y);
            } else {
              const bool hi = lane & Cfg::TASKS;
              float h[2][4];   // rows 2 hi + r
  #pragma unroll
              for (int r = 0; r < 2; ++r)
  #pragma unroll
                for (int b = 0; b < 4; ++b) {
                  const float send = hi ? pair_at(acc[r], b) : pair_at(acc[r + 2], b);
                  const float keep = hi ? pair_at(acc[r + 2], b) : pair_at(acc[r], b);
                  h[r][b] = keep + __shfl_xor_sync(0xffffffffu, send, Cfg::TASKS);
                }
              if constexpr (Cfg::PW == 2) {
  #pragma unroll
                for (int r = 0; r < 2; ++r)
                  *reinterpret_cast<float4*>(dst + (4 * jb + 2 * hi + r) * DP) =
                      make_float4(h[r][0], h[r][1], h[r][2], h[r][3]);
              } else {
                const bool hi2 = lane & (2 * Cfg::TASKS);
  #pragma unroll
                for (int r = 0; r < 2; ++r) {
                  float q2[2];   // columns 2 hi2 + b
  #pragma unroll
                  for (int b = 0; b < 2; ++b) {
                    const float send = hi2 ? h[r][b] : h[r][b + 2];
                    const float keep = hi2 ? h[r][b + 2] : h[r][b];
                    q2[b] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * Cfg::TASKS);
                  }
                  *reinterpret_cast<float2*>(dst + (4 * jb + 2 * hi + r) * DP + 2 * hi2) =
                      make_float2(q2[0], q2[1]);
                }
              }
            }
          }
        }

        // phase 2b: per Gaussian sums over pixels (G threads per Gaussian, consecutive lanes)
        if constexpr (!FO) {
          constexpr int G = Cfg::G;
          const int j = t / G, pg = t % G;
          // moments of dL/do (so = its sum); those of dL/dsigma are -o times these
          float mx = 0.f, my = 0.f, mxx = 0.f, mxy = 0.f, myy = 0.f;
          float so = 0.f, sr = 0.f, sg = 0.f, sb = 0.f, sz = 0.f;
          // strip by strip: the G lanes of Gaussian j skip whole strips it cannot reach
          constexpr int PPS = 32 / G;   // pixels per strip per lane
          static_assert(G == 16 && kStripW == 8 && kStripH == 4, "pixel offsets below");
          // pixel q = 32 ws + pg + 16 u lies at column 8 (ws & 1) + (pg & 7) and row
          // 4 (ws >> 1) + (pg >> 3) + 2 u of the tile (strip_px / strip_py of q)
          const float xl = (float)(pg & 7) - 7.5f, yl = (float)(pg >> 3) - 7.5f;
  #pragma unroll
          for (int ws = 0; ws < kT / 32; ++ws) {
            if (!(s_live[ws] >> j & 1u)) continue;   // uniform over the G lanes of j
  #pragma unroll
            for (int u = 0; u < PPS; ++u) {
            const int q = ws * 32 + pg + u * G;
            const float w = s_W[j * kWS + q], go = s_GO[j * kWS + q];
            const float4 e = s_E4[q];
            const float x = xl + (float)(8 * (ws & 1)), y = yl + (float)(4 * (ws >> 1) + 2 * u);
            mx = fmaf(go, x, mx);
            my = fmaf(go, y, my);
            mxx = fmaf(go * x, x, mxx);
            mxy = fmaf(go * x, y, mxy);
            myy = fmaf(go * y, y, myy);
            so += go;
            sr = fmaf(w, e.x, sr);
            sg = fmaf(w, e.y, sg);
            sb = fmaf(w, e.z, sb);
            sz = fmaf(w, e.w, sz);
            }
          }
          // the ten sums over the G = 16 lanes of Gaussian j by a reduce-scatter (each level
          // halves the values a lane carries: 5 + 3 + 2 + 1 shuffles instead of 4 x 10), then
          // every lane reads the ten totals from the lanes holding them (0 1 2 4 5 8 9 10 12 13)
          static_assert(G == 16, "the reduce-scatter is laid out for 16 lanes per Gaussian");
          {
            const float v[10] = {mx, my, mxx, mxy, myy, so, sr, sg, sb, sz};
            float r1[6], r2[4], r3[2];
  #pragma unroll
            for (int k = 0; k < 5; ++k) {
              const bool hi = pg & 8;
              const float send = hi ? v[k] : v[k + 5], keep = hi ? v[k + 5] : v[k];
              r1[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            r1[5] = 0.f;
  #pragma unroll
            for (int k = 0; k < 3; ++k) {
              const bool hi = pg & 4;
              const float send = hi ? r1[k] : r1[k + 3], keep = hi ? r1[k + 3] : r1[k];
              r2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            r2[3] = 0.f;
  #pragma unroll
            for (int k = 0; k < 2; ++k) {
              const bool hi = pg & 2;
              const float send = hi ? r2[k] : r2[k + 2], keep = hi ? r2[k + 2] : r2[k];
              r3[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
            const bool hi = pg & 1;
            const float r4 = (hi ? r3[1] : r3[0]) + __shfl_xor_sync(0xffffffffu, hi ? r3[0] : r3[1], 1);
            const int base = lane & 16;
            mx = __shfl_sync(0xffffffffu, r4, base + 0);
            my = __shfl_sync(0xffffffffu, r4, base + 1);
            mxx = __shfl_sync(0xffffffffu, r4, base + 2);
            mxy = __shfl_sync(0xffffffffu, r4, base + 4);
            myy = __shfl_sync(0xffffffffu, r4, base + 5);
            so = __shfl_sync(0xffffffffu, r4, base + 8);
            sr = __shfl_sync(0xffffffffu, r4, base + 9);
            sg = __shfl_sync(0xffffffffu, r4, base + 10);
            sb = __shfl_sync(0xffffffffu, r4, base + 12);
            sz = __shfl_sync(0xffffffffu, r4, base + 13);
          }
          if (pg == 0 && j < bc) {
            const float4 r0 = s_r0[jb0 + j];
            const float4 r1 = s_r1[jb0 + j];
            // moments are about the tile centre: pixel offset dx = x - uc with uc = u - centre
            const float uc = r0.x - ((float)tx0 + 8.f), vc = r0.y - ((float)ty0 + 8.f);
            const float A = r0.z, Bq = r0.w, C = r1.x;
            const float no = -r1.y;                                        // -o
            const float m1 = no * so;
            mx *= no;
            my *= no;
            mxx *= no;
            mxy *= no;
            myy *= no;
            const float sdx = mx - uc * m1, sdy = my - vc * m1;            // sum gs dx, sum gs dy
            const float sdxx = mxx - 2.f * uc * mx + uc * uc * m1;         // sum gs dx^2
            const float sdyy = myy - 2.f * vc * my + vc * vc * m1;
            const float sdxy = mxy - uc * my - vc * mx + uc * vc * m1;
            const float gAq = 0.5f * sdxx, gBq = sdxy, gCq = 0.5f * sdyy;
            const float gu = -(A * sdx + Bq * sdy), gv = -(C * sdy + Bq * sdx);
            float* dst = g2d + (int64_t)s_id[jb0 + j] * kG2D;
            red_add4(dst, gu, gv, gAq, gBq);
            red_add4(dst + 4, gCq, so, sr, sg);
            red_add4(dst + 8, sb, sz, 0.f, 0.f);
          }
        }
        if constexpr (DP > 0 && !FO) {
          if (more) fb.store(D, s_fb + ((bi + 1) & 1) * B * DP);
        }
        __syncthreads();

        // flush the batch's feature-gradient sums (the partials added in order)
        if constexpr (DP > 0) {
          if (g_feats) {
            constexpr int NP = Cfg::NPART;
            if (D == DP) {
              for (int e = t; e < bc * (DP / 4); e += kT) {
                const int j = e / (DP / 4), q = e - j * (DP / 4);
                float4* so = reinterpret_cast<float4*>(s_outF + j * DP + 4 * q);
                float4 v = *so;
  #pragma unroll
                for (int w = 1; w < NP; ++w) {
                  const float4 u = so[w * (B * DP / 4)];
                  v.x += u.x;
                  v.y += u.y;
                  v.z += u.z;
                  v.w += u.w;
                }
                atomicAdd(reinterpret_cast<float4*>(g_feats + (int64_t)s_id[jb0 + j] * D + 4 * q), v);
              }
            } else {
              for (int e = t; e < bc * DP; e += kT) {
                const int j = e / DP, c = e - j * DP;
                float v = s_outF[e];
  #pragma unroll
                for (int w = 1; w < NP; ++w) v += s_outF[w * (B * DP) + e];
                if (c < D) atomicAdd(g_feats + (int64_t)s_id[jb0 + j] * D + c, v);
              }
            }
          }
        }
      }
    }
    }
    __syncthreads();   // shared memory and s_tile are reused by the next tile
  }
}

template <int DP, bool BF16, bool FO, int NJ>
void launch_t(const RasterJobs<NJ>& jobs, const TileQueue& tq, cudaStream_t st) {
  const size_t smem = sizeof(float) * BwdCfg<DP, FO>::smem_floats;
  auto kern = k_raster_bwd<DP, BF16, FO, NJ>;
  const int items = jobs.job[NJ > 1 ? jobs.n - 1 : 0].item_end;
  const int grid = persistent_grid(kern, kT, smem, items);
  kern<<<grid, kT, smem, st>>>(jobs, tq);
  note_launch();
}

// Dispatch of the run-time options to the kernel variants (features-only needs features).
template <int DP>
void launch_dp(bool bf, bool fo, const RasterJobs<1>& jobs, const TileQueue& tq, cudaStream_t st) {
  if constexpr (DP > 0) {
    if (fo) {
      if (bf)
        launch_t<DP, true, true, 1>(jobs, tq, st);
      else
        launch_t<DP, false, true, 1>(jobs, tq, st);
      return;
    }
  }
  if (bf)
    launch_t<DP, true, false, 1>(jobs, tq, st);
  else
    launch_t<DP, false, false, 1>(jobs, tq, st);
}

template <int DP>
void launch_dp_jobs(bool bf, const RasterJobs<kMaxJobs>& jobs, const TileQueue& tq, cudaStream_t st) {
  if (bf)
    launch_t<DP, true, false, kMaxJobs>(jobs, tq, st);
  else
    launch_t<DP, false, false, kMaxJobs>(jobs, tq, st);
}

}  // namespace

void launch_raster_bwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec,
                       const void* feats, int feat_dtype, int D, const uint2* ranges,
                       const uint32_t* inst_id, const float* T_final, const uint32_t* n_contrib,
                       const float* g_rgb, const float* g_depth, const float* g_alpha,
                       const float* g_feat, float* g2d, float* g_feats, bool features_only,
                       cudaStream_t st) {
  if (cam.TX * cam.TY == 0) return;
  const bool bf = feat_dtype == GS_BF16;
  const int DP = g_feat ? padded_feat(D) : 0;
  const bool fo = features_only && DP > 0 && g_feats;
  RasterJobs<1> jobs{};
  jobs.n = 1;
  RasterJob& j = jobs.job[0];
  j.cam = cam;
  j.rec = rec;
  j.feats = feats;
  j.D = D;
  j.item_end = tq.n_tiles;
  j.ranges = ranges;
  j.inst_id = inst_id;
  j.order = tq.order;
  j.T_final = const_cast<float*>(T_final);
  j.n_contrib = const_cast<uint32_t*>(n_contrib);
  j.g_rgb = g_rgb;
  j.g_depth = g_depth;
  j.g_alpha = g_alpha;
  j.g_feat = g_feat;
  j.g2d = g2d;
  j.g_feats = g_feats;
#define GS_BWD(dp) launch_dp<dp>(bf, fo, jobs, tq, st)
  switch (DP) {
    case 0: GS_BWD(0); break;
    case 8: GS_BWD(8); break;
    case 16: GS_BWD(16); break;
    case 32: GS_BWD(32); break;
    default: GS_BWD(64); break;
  }
#undef GS_BWD
}

void launch_raster_bwd_jobs(const RasterJob* src, int n, int feat_dtype, bool want_feat,
                            const TileQueue& tq, cudaStream_t st) {
  if (n <= 0 || n > kMaxJobs) return;
  RasterJobs<kMaxJobs> jobs{};
  jobs.n = n;
  int Dmax = 0;
  for (int k = 0; k < n; ++k) {
    jobs.job[k] = src[k];
    Dmax = std::max(Dmax, src[k].D);
  }
  if (jobs.job[n - 1].item_end <= 0) return;
  const bool bf = feat_dtype == GS_BF16;
  const int DP = want_feat ? padded_feat(Dmax) : 0;
#define GS_BWD(dp) launch_dp_jobs<dp>(bf, jobs, tq, st)
  switch (DP) {
    case 0: GS_BWD(0); break;
    case 8: GS_BWD(8); break;
    case 16: GS_BWD(16); break;
    case 32: GS_BWD(32); break;
    default: GS_BWD(64); break;
  }
#undef GS_BWD
}

}  // namespace gs
