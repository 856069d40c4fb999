// a3: forward rendering, X-GS Eq. 1 (front-to-back alpha blending over depth-sorted
// Gaussians), depth by substituting c_i -> d_i (App. B) and features by c_i -> f_i
// (Sec. 3.1).  One 128-thread CTA per half tile (16 x 8 pixels), one thread per pixel:
// both halves walk the tile's list, each culling it against its own pixel box, which
// halves the longest work item (the tail of the persistent schedule).
//
// The tile's sorted list is consumed in batches of 128 Gaussians staged in shared
// memory (records gathered by id; features converted to fp32 once per batch, so bf16
// storage costs no per-pixel conversion).  Each warp owns an 8 x 4 pixel strip and visits
// only the batch entries that can reach it (ballot over a per-strip box test), stops when
// all its pixels have terminated (checked before each group of 32 candidates), and the
// CTA stops when all 128 pixels have.  The walk is software-pipelined by one entry: the
// colour, depth and feature terms of an entry are added while the next entry's opacity is
// evaluated, so the accumulation and the evaluation chain overlap in one warp.
#include <algorithm>

#include "gs_blend.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kB = 128;    // batch = threads = pixels per work item (part of a tile)
constexpr int kRowsB = kB / 16;            // pixel rows per work item
constexpr int kSplit = kTilePix / kB;      // work items per tile

template <int DP, bool BF16>
__device__ __forceinline__ void stage_features(const void* __restrict__ feats, int D,
                                               const uint32_t* __restrict__ s_id, int cnt,
                                               float* __restrict__ s_feat) {
  if constexpr (DP > 0) {
    if (D == DP) {
      // 16-byte chunks: 8 bf16 or 4 f32 values
      constexpr int VPC = BF16 ? 8 : 4;
      constexpr int CPR = DP / VPC;
      for (int c = threadIdx.x; c < cnt * CPR; c += kB) {
        const int j = c / CPR, part = c - j * CPR;
        const int64_t row = (int64_t)s_id[j] * DP;
        float* dst = s_feat + j * DP + part * VPC;
        if constexpr (BF16) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(
              static_cast<const __nv_bfloat16*>(feats) + row) + part);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            dst[2 * k] = __uint_as_float(w[k] << 16);
            dst[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
          }
        } else {
          const float4 v = __ldg(reinterpret_cast<const float4*>(
              static_cast<const float*>(feats) + row) + part);
          *reinterpret_cast<float4*>(dst) = v;
        }
      }
    } else {
      for (int e = threadIdx.x; e < cnt * DP; e += kB) {
        const int j = e / DP, c = e - j * DP;
        float v = 0.f;
        if (c < D) {
          const int64_t idx = (int64_t)s_id[j] * D + c;
          if constexpr (BF16)
            v = __bfloat162float(static_cast<const __nv_bfloat16*>(feats)[idx]);
          else
            v = __ldg(static_cast<const float*>(feats) + idx);
        }
        s_feat[e] = v;
      }
    }
  }
}

// Resident CTAs per SM by channel count, the most whose register share (80, 96, 128) holds
// the kernel without spills: 6 up to 16 channels, 5 at 32, 4 at 64.
static_assert(kSplit == kFwdItemsPerTile, "work items per tile");

// J: the renders of this launch (one for a plain render, up to kMaxJobs for a serving
// batch); their half tiles are taken from one queue.
template <int DP, bool BF16, bool LOSS, int NJ>
__global__ void __launch_bounds__(kB, DP <= 16 ? 6 : (DP <= 32 ? 5 : 4))
k_raster_fwd(const __grid_constant__ RasterJobs<NJ> J, TileQueue tq, FeatLoss fl) {
  __shared__ float4 s_r0[kB], s_r1[kB], s_r2[kB];
  __shared__ uint32_t s_id[kB];
  __shared__ int s_orig[kB];
  __shared__ int s_wc[kB / 32];
  __shared__ int s_tile, s_job;
  extern __shared__ __align__(16) float s_feat[];   // [kB][DP]
  double l1_sum = 0.0, cos_sum = 0.0;   // fused loss (LOSS): this thread's samples, all tiles

  // persistent CTA: tiles from the queue, heaviest first
  for (;;) {
    if (threadIdx.x == 0) {
      // work item q: part (local mod kSplit) of the (local / kSplit)-th tile of its job in
      // heavy-first order, local = q - the job's first item
      const uint32_t q = atomicAdd(tq.head, 1u);
      s_tile = -1;
      if (q < J.items()) {
        uint32_t first;
        const int k = J.find(q, &first);
        const uint32_t local = q - first, r = local / kSplit;
        const uint32_t* order = J.job[k].order;
        s_tile = kSplit * (int)(order ? order[r] : r) + (int)(local - r * kSplit);
        s_job = k;
      }
    }
    __syncthreads();
    const int item = s_tile;
    if (item < 0) break;
    const RasterJob& jb = J.job[NJ > 1 ? s_job : 0];
    const CamDev& cam = jb.cam;
    const GaussRec* __restrict__ rec = jb.rec;
    const void* __restrict__ feats = jb.feats;
    const int D = jb.D;
    const uint2* __restrict__ ranges = jb.ranges;
    const uint32_t* __restrict__ inst_id = jb.inst_id;
    const int tile = item / kSplit;

    const int tx0 = (tile % cam.TX) * kTile, ty0 = (tile / cam.TX) * kTile + kRowsB * (item % kSplit);
    const int px = tx0 + strip_px(threadIdx.x);
    const int py = ty0 + strip_py(threadIdx.x);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    const int start = (int)rg.x, end = (int)rg.y;
    const int lane = threadIdx.x & 31;
    // pixel-centre boxes of the work item and of this warp's 8 x 4 strip
    const float bx0 = (float)tx0 + 0.5f, by0 = (float)ty0 + 0.5f;
    const float wbx0 = (float)(tx0 + strip_px(threadIdx.x & ~31)) + 0.5f;
    const float wby0 = (float)(ty0 + strip_py(threadIdx.x & ~31)) + 0.5f;

    float T = 1.f;
    float2 c01 = make_float2(0.f, 0.f), c2d = make_float2(0.f, 0.f);   // (r, g), (b, depth)
    float2 acc[DP > 0 ? DP / 2 : 1];   // feature channels in packed pairs
#pragma unroll
    for (int c = 0; c < (DP > 0 ? DP / 2 : 1); ++c) acc[c] = make_float2(0.f, 0.f);
    int last = 0;     // 1 + list position of the last blended entry
    int lastj = -1;   // its batch slot, resolved to a list position once per batch
    bool done = !inside;
    int pj = -1;      // entry whose terms are still to be added (software pipeline)
    float pw = 0.f;   // its weight for this pixel (0 where it does not blend)
    float pz = 0.f;   // its depth
    auto accumulate = [&](int j, float w, float z) {
      const float4 r2 = s_r2[j];
      const float2 w2 = splat2(w);
      c01 = fma2(w2, make_float2(r2.x, r2.y), c01);
      c2d = fma2(w2, make_float2(r2.z, z), c2d);
      if constexpr (DP > 0) {
        const float4* f4 = reinterpret_cast<const float4*>(s_feat + j * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
          const float4 f = f4[q];
          acc[2 * q] = fma2(w2, make_float2(f.x, f.y), acc[2 * q]);
          acc[2 * q + 1] = fma2(w2, make_float2(f.z, f.w), acc[2 * q + 1]);
        }
      }
    };

    for (int b0 = start; b0 < end; b0 += kB) {
      if (__syncthreads_count(done) == kB) break;
      const int cnt = min(kB, end - b0);
      // gather the batch and drop entries that no pixel of this tile can blend
      bool keep = false;
      uint32_t id = 0;
      GaussRec g;
      if ((int)threadIdx.x < cnt) id = inst_id[b0 + threadIdx.x];
      if ((int)threadIdx.x < cnt && id < (uint32_t)cam.n_gauss) {
        g = rec[id];
        g.r1.w = sigma_cut(g.r1.y);
        keep = box_min_sigma(bx0, by0, bx0 + 15.f, by0 + (float)(kRowsB - 1), g.r0.x, g.r0.y,
                             g.r0.z, g.r0.w, g.r1.x) <= g.r1.w;
      }
      int nk;
      const int pos = block_compact_index<kB / 32>(keep, s_wc, &nk);
      if (keep) {
        s_r0[pos] = g.r0;
        s_r1[pos] = g.r1;      // r1.w = sigma cut
        s_r2[pos] = g.r2;
        s_id[pos] = id;
        s_orig[pos] = b0 + (int)threadIdx.x - start;
      }
      __syncthreads();
      stage_features<DP, BF16>(feats, D, s_id, nk, s_feat);
      __syncthreads();
      // each warp (an 8 x 4 pixel strip) visits only the entries that can reach its strip:
      // the lanes test 32 entries at a time and the ballot lists the survivors
      for (int g0 = 0; g0 < nk; g0 += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        bool hit = false;
        if (g0 + lane < nk) {
          const float4 q0 = s_r0[g0 + lane], q1 = s_r1[g0 + lane];
          hit = box_min_sigma(wbx0, wby0, wbx0 + (float)(kStripW - 1), wby0 + (float)(kStripH - 1),
                              q0.x, q0.y, q0.z, q0.w, q1.x) <= q1.w;
        }
        unsigned live = __ballot_sync(0xffffffffu, hit);
        while (live) {
          const int j = g0 + __ffs(live) - 1;
          live &= live - 1;
          const float4 r0 = s_r0[j];
          const float4 r1 = s_r1[j];
          const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
          const float a = fminf(kAlphaMax, __fmul_rn(r1.y, blend_gauss(sigma)));
          // the previous entry is accumulated while this one's opacity is evaluated (the
          // two are independent; each pixel still adds its terms in list order)
          if (pj >= 0) accumulate(pj, pw, pz);
          float w = 0.f;
          if (!done && sigma >= 0.f && sigma <= r1.w && a >= kAlphaMin) {
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
            if (Tn < kTMin) {
              done = true;
            } else {
              w = __fmul_rn(a, T);
              T = Tn;
              lastj = j;
            }
          }
          pj = j;
          pw = w;
          pz = r1.z;
        }
      }
      if (pj >= 0) accumulate(pj, pw, pz);   // before the batch's features are replaced
      pj = -1;
      if (lastj >= 0) { last = s_orig[lastj] + 1; lastj = -1; }
    }
    if (inside) {
      float *rgb = jb.rgb, *depth = jb.depth, *alpha = jb.alpha, *feat = jb.feat;
      const int64_t HW = (int64_t)cam.W * cam.H;
      const int64_t p = (int64_t)py * cam.W + px;
      if (rgb) {
        rgb[p] = c01.x;
        rgb[HW + p] = c01.y;
        rgb[2 * HW + p] = c2d.x;
      }
      if (depth) depth[p] = c2d.y;
      if (alpha) alpha[p] = 1.f - T;
      if constexpr (DP > 0) {
        if (feat) {
#pragma unroll
          for (int c = 0; c < DP; ++c)
            if (c < D) feat[c * HW + p] = pair_at(acc, c);
        }
      }
      jb.T_final[p] = T;
      jb.n_contrib[p] = (uint32_t)last;
    }
    if constexpr (LOSS) {
      // Masked L1 + cosine loss of each sample and its gradient w.r.t. G_hat.  The
      // target column is parked in the (now idle) feature staging area, so that neither
      // the target nor the rendered features need a second register copy.
      __syncthreads();   // every warp is done with the batch features in s_feat
      if (inside) {
        const int64_t HW = (int64_t)cam.W * cam.H;
        const int64_t p = (int64_t)py * cam.W + px;
        const float V = fl.mask ? __ldg(fl.mask + p) : 1.f;
        float dot = 0.f, aa = 0.f, bb = 0.f, l1 = 0.f;
#pragma unroll
        for (int c = 0; c < DP; ++c) {
          if (c < D) {
            const float a = V * pair_at(acc, c), b = V * __ldg(fl.target + c * HW + p);
            s_feat[c * kB + threadIdx.x] = b;
            dot = fmaf(a, b, dot);
            aa = fmaf(a, a, aa);
            bb = fmaf(b, b, bb);
            l1 += fabsf(a - b);
          }
        }
        const float la = sqrtf(aa), lb = sqrtf(bb);
        const float inv = 1.f / (fmaxf(la, kCosEps) * fmaxf(lb, kCosEps));
        const float cosv = dot * inv;
        const float cf = la > kCosEps ? cosv / aa : 0.f;   // d cos / da = b inv - cos a / |a|^2
#pragma unroll
        for (int c = 0; c < DP; ++c) {
          if (c < D) {
            const float a = V * pair_at(acc, c), b = s_feat[c * kB + threadIdx.x];
            const float sg = a > b ? 1.f : (a < b ? -1.f : 0.f);
            fl.g_feat[c * HW + p] = V * (fl.w_l1 * sg - fl.w_cos * (b * inv - cf * a));
          }
        }
        l1_sum += (double)l1;
        cos_sum += (double)(1.f - cosv);
      }
    }
    __syncthreads();   // shared memory and s_tile are reused by the next tile
  }
  if (threadIdx.x == 0) queue_leave(tq, gridDim.x);
  if constexpr (LOSS) {
    {
      // one block reduction and three atomics per CTA for the whole launch
      __shared__ double s_red[2][kB / 32];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, o);
        cos_sum += __shfl_xor_sync(0xffffffffu, cos_sum, o);
      }
      if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = l1_sum;
        s_red[1][threadIdx.x >> 5] = cos_sum;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kB / 32; ++w) {
          a += s_red[0][w];
          b += s_red[1][w];
        }
        a *= fl.s_l1;
        b *= fl.s_cos;
        atomicAdd(fl.loss, fl.lambda * (a + b));
        atomicAdd(fl.loss + 1, a);
        atomicAdd(fl.loss + 2, b);
      }
    }
  }
}

template <int DP, bool BF16, bool LOSS, int NJ>
void launch_t(const RasterJobs<NJ>& jobs, const TileQueue& tq, const FeatLoss& fl, cudaStream_t st) {
  const size_t smem = sizeof(float) * kB * DP;
  auto kern = k_raster_fwd<DP, BF16, LOSS, NJ>;
  const int items = jobs.job[NJ > 1 ? jobs.n - 1 : 0].item_end;
  const int grid = persistent_grid(kern, kB, smem, items);
  kern<<<grid, kB, smem, st>>>(jobs, tq, fl);
  note_launch();
}

// Dispatch of the run-time options to the kernel variants (the loss needs features).
template <int DP>
void launch_dp(bool bf, bool loss, const RasterJobs<1>& jobs, const TileQueue& tq,
               const FeatLoss& fl, cudaStream_t st) {
  if constexpr (DP > 0) {
    if (loss) {
      if (bf)
        launch_t<DP, true, true, 1>(jobs, tq, fl, st);
      else
        launch_t<DP, false, true, 1>(jobs, tq, fl, st);
      return;
    }
  }
  if (bf)
    launch_t<DP, true, false, 1>(jobs, tq, fl, st);
  else
    launch_t<DP, false, false, 1>(jobs, tq, fl, st);
}

template <int DP>
void launch_dp_jobs(bool bf, const RasterJobs<kMaxJobs>& jobs, const TileQueue& tq, cudaStream_t st) {
  const FeatLoss fl{};
  if (bf)
    launch_t<DP, true, false, kMaxJobs>(jobs, tq, fl, st);
  else
    launch_t<DP, false, false, kMaxJobs>(jobs, tq, fl, st);
}

}  // namespace

int padded_feat(int D) {
  if (D <= 0) return 0;
  if (D <= 8) return 8;
  if (D <= 16) return 16;
  if (D <= 32) return 32;
  return 64;
}

void launch_raster_fwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec,
                       const void* feats, int feat_dtype, int D, const uint2* ranges,
                       const uint32_t* inst_id, float* rgb, float* depth, float* alpha, float* feat,
                       float* T_final, uint32_t* n_contrib, const FeatLoss* loss,
                       cudaStream_t st) {
  if (cam.TX * cam.TY == 0) return;
  const bool bf = feat_dtype == GS_BF16;
  FeatLoss fl{};
  if (loss && D > 0) fl = *loss;
  // features are blended when written or when the fused loss needs them
  const int DP = (feat || fl.target) ? padded_feat(D) : 0;
  const bool loss_on = fl.target != nullptr;
  RasterJobs<1> jobs{};
  jobs.n = 1;
  RasterJob& j = jobs.job[0];
  j.cam = cam;
  j.rec = rec;
  j.feats = feats;
  j.D = D;
  j.item_end = kSplit * tq.n_tiles;
  j.ranges = ranges;
  j.inst_id = inst_id;
  j.order = tq.order;
  j.rgb = rgb;
  j.depth = depth;
  j.alpha = alpha;
  j.feat = feat;
  j.T_final = T_final;
  j.n_contrib = n_contrib;
#define GS_FWD(dp) launch_dp<dp>(bf, loss_on, jobs, tq, fl, st)
  switch (DP) {
    case 0: GS_FWD(0); break;
    case 8: GS_FWD(8); break;
    case 16: GS_FWD(16); break;
    case 32: GS_FWD(32); break;
    default: GS_FWD(64); break;
  }
#undef GS_FWD
}

void launch_raster_fwd_jobs(const RasterJob* src, int n, int feat_dtype, bool want_feat,
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
#define GS_FWD(dp) launch_dp_jobs<dp>(bf, jobs, tq, st)
  switch (DP) {
    case 0: GS_FWD(0); break;
    case 8: GS_FWD(8); break;
    case 16: GS_FWD(16); break;
    case 32: GS_FWD(32); break;
    default: GS_FWD(64); break;
  }
#undef GS_FWD
}

}  // namespace gs
