// Rendering on a stride-s sample grid (grid-sampled supervision, X-GS Sec. 3.2 and App. D):
// only the samples (u, v) = (o_h + m s, o_w + n s) are rendered, into a compact
// ceil(H/s) x ceil(W/s) map, each equal to the full-resolution render at its pixel.
//
// Gaussians stay binned in 16x16 image tiles (the same lists as a full render), so a
// sample blends exactly the Gaussians its pixel would.  An image tile holds only
// ceil(16/s)^2 samples (64 at s = 2, 16 at s = 4), too few for a 256-thread tile CTA, so
// the work item is (image tile, chunk of up to 32 of its samples) and each warp runs one
// item at a time: it walks the tile's depth-sorted list in batches of 32 entries, culls
// them against the box of its samples, stages the survivors (records and features) in
// its own slice of shared memory and blends them into one sample per lane.  Warps pull
// items from a queue in heavy-first tile order; per sample the work is the tile's list,
// so the grid costs about 1/s^2 of a full render plus one pass over the lists.
//
// The backward replays transmittance in reverse per lane (as the tile kernel does), sums
// each Gaussian's per-sample terms with warp shuffles, and forms the feature gradient
// W^T g_F of each batch in shared memory.  Samples that fall outside the image (large
// offsets) are written by a separate fill kernel.
#include "gs_blend.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kGT = 256;           // threads per CTA: 8 independent warps
constexpr int kWarps = kGT / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWT = 32;            // row stride of the per-warp weight matrix [lane][entry]

// Position of entry k in lane l's row of the weight matrix: 16-byte chunks XOR-swizzled by
// the lane, so that the 32 lanes' stores of one entry spread over 8 banks and a 16-byte
// read of four consecutive entries stays contiguous.
__device__ __forceinline__ int w_slot(int l, int k) {
  return l * kWT + ((((k >> 2) ^ (l & 7)) << 2) | (k & 3));
}

__device__ __forceinline__ int ceil_div_signed(int a, int b) {   // b > 0
  return a >= 0 ? (a + b - 1) / b : -((-a) / b);
}

// Samples of image tile (tx, ty): columns [n0, n1), rows [m0, m1) of the compact grid.
struct TileSamples {
  int n0, n1, m0, m1;
};

__device__ __forceinline__ TileSamples tile_samples(const CamDev& c, int tx, int ty) {
  TileSamples t;
  t.n0 = max(0, ceil_div_signed(16 * tx - c.ox, c.stride));
  t.n1 = min(c.GW, ceil_div_signed(16 * tx + 16 - c.ox, c.stride));
  t.m0 = max(0, ceil_div_signed(16 * ty - c.oy, c.stride));
  t.m1 = min(c.GH, ceil_div_signed(16 * ty + 16 - c.oy, c.stride));
  return t;
}

// One work item as seen by a lane: its sample and pixel.
struct ItemLane {
  int tile;
  int n, m;        // compact sample
  int px, py;      // image pixel
  bool in_img;     // a sample of this item inside the image
  float bx0, by0, bx1, by1;   // box of the item's sample centres (warp-uniform)
};

__device__ __forceinline__ bool decode_item(const CamDev& cam, const TileQueue& tq, int CH,
                                            uint32_t q, ItemLane* it) {
  const int lane = threadIdx.x & 31;
  const int rank = (int)(q / (uint32_t)CH), chunk = (int)(q - (uint32_t)rank * CH);
  const int tile = tq.order ? (int)tq.order[rank] : rank;
  const TileSamples ts = tile_samples(cam, tile % cam.TX, tile / cam.TX);
  const int cx = max(0, ts.n1 - ts.n0), cy = max(0, ts.m1 - ts.m0);
  const int k = chunk * 32 + lane;
  const bool valid = k < cx * cy;
  it->tile = tile;
  it->n = valid ? ts.n0 + k % cx : 0;
  it->m = valid ? ts.m0 + k / cx : 0;
  it->px = grid_coord(cam.ox, cam.stride, it->n);
  it->py = grid_coord(cam.oy, cam.stride, it->m);
  it->in_img = valid && it->px < cam.W && it->py < cam.H;
  if (!__any_sync(kFull, it->in_img)) return false;
  float x0 = it->in_img ? (float)it->px + 0.5f : 3.0e38f, x1 = it->in_img ? (float)it->px + 0.5f : -3.0e38f;
  float y0 = it->in_img ? (float)it->py + 0.5f : 3.0e38f, y1 = it->in_img ? (float)it->py + 0.5f : -3.0e38f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(kFull, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(kFull, x1, o));
    y0 = fminf(y0, __shfl_xor_sync(kFull, y0, o));
    y1 = fmaxf(y1, __shfl_xor_sync(kFull, y1, o));
  }
  it->bx0 = x0;
  it->bx1 = x1;
  it->by0 = y0;
  it->by1 = y1;
  return true;
}

__device__ __forceinline__ uint32_t next_item(uint32_t* head) {
  uint32_t q = 0;
  if ((threadIdx.x & 31) == 0) q = atomicAdd(head, 1u);
  return __shfl_sync(kFull, q, 0);
}

// Gather entries [b0, b0 + 32) of a tile list (up to `end`), keep those that can reach the
// item's box, and compact them in list order into the warp's staging slots.  Returns the
// number kept.
__device__ __forceinline__ int stage_batch(const CamDev& cam, const ItemLane& it,
                                           const GaussRec* __restrict__ rec,
                                           const uint32_t* __restrict__ inst_id, int b0, int end,
                                           int start, float4* s_r, uint32_t* s_id, int* s_orig) {
  const int lane = threadIdx.x & 31;
  const int j = b0 + lane;
  bool keep = false;
  uint32_t id = 0;
  GaussRec g;
  if (j < end) {
    id = inst_id[j];
    if (id < (uint32_t)cam.n_gauss) {
      g = rec[id];
      g.r1.w = sigma_cut(g.r1.y);
      keep = box_min_sigma(it.bx0, it.by0, it.bx1, it.by1, g.r0.x, g.r0.y, g.r0.z, g.r0.w, g.r1.x) <=
             g.r1.w;
    }
  }
  const unsigned km = __ballot_sync(kFull, keep);
  if (keep) {
    const int pos = __popc(km & ((1u << lane) - 1u));
    s_r[3 * pos] = g.r0;
    s_r[3 * pos + 1] = g.r1;   // r1.w = sigma cut
    s_r[3 * pos + 2] = g.r2;
    s_id[pos] = id;
    s_orig[pos] = j - start;
  }
  return __popc(km);
}

// Features of the nk staged entries, widened to fp32: s_f[k][DP].
template <int DP, bool BF16>
__device__ __forceinline__ void stage_feats(const void* __restrict__ feats, int D,
                                            const uint32_t* s_id, int nk, float* s_f) {
  const int lane = threadIdx.x & 31;
  if (D == DP) {
    constexpr int VPC = BF16 ? 8 : 4;
    constexpr int CPR = DP / VPC;
    for (int c = lane; c < nk * CPR; c += 32) {
      const int k = c / CPR, part = c - k * CPR;
      const int64_t row = (int64_t)s_id[k] * DP;
      float* dst = s_f + k * DP + part * VPC;
      if constexpr (BF16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(feats) + row) + part);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          dst[2 * e] = __uint_as_float(w[e] << 16);
          dst[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
        }
      } else {
        *reinterpret_cast<float4*>(dst) =
            __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(feats) + row) + part);
      }
    }
  } else {
    for (int e = lane; e < nk * DP; e += 32) {
      const int k = e / DP, c = e - k * DP;
      float v = 0.f;
      if (c < D) {
        const int64_t idx = (int64_t)s_id[k] * D + c;
        if constexpr (BF16)
          v = __bfloat162float(static_cast<const __nv_bfloat16*>(feats)[idx]);
        else
          v = __ldg(static_cast<const float*>(feats) + idx);
      }
      s_f[e] = v;
    }
  }
}

template <int DP>
constexpr int fwd_warp_floats() {
  return 32 * 12 + 32 + 32 + 32 * DP;   // records, ids, list positions, features
}

template <int DP, bool BF16, bool LOSS>
__global__ void __launch_bounds__(kGT, 2)
k_grid_fwd(CamDev cam, TileQueue tq, int CH, const GaussRec* __restrict__ rec,
           const void* __restrict__ feats, int D, const uint2* __restrict__ ranges,
           const uint32_t* __restrict__ inst_id, float* __restrict__ rgb, float* __restrict__ depth,
           float* __restrict__ alpha, float* __restrict__ feat, float* __restrict__ T_final,
           uint32_t* __restrict__ n_contrib, FeatLoss fl) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* base = smem + warp * fwd_warp_floats<DP>();
  float4* s_r = reinterpret_cast<float4*>(base);
  uint32_t* s_id = reinterpret_cast<uint32_t*>(base + 32 * 12);
  int* s_orig = reinterpret_cast<int*>(base + 32 * 12 + 32);
  float* s_f = base + 32 * 12 + 64;
  const int64_t HW = (int64_t)cam.GW * cam.GH;
  double l1_sum = 0.0, cos_sum = 0.0;

  for (;;) {
    const uint32_t q = next_item(tq.head);
    if (q >= (uint32_t)tq.n_tiles) break;
    ItemLane it;
    if (!decode_item(cam, tq, CH, q, &it)) continue;
    const float fx = (float)it.px + 0.5f, fy = (float)it.py + 0.5f;
    const uint2 rg = ranges[it.tile];
    const int start = (int)rg.x, end = (int)rg.y;

    float T = 1.f;
    float2 c01 = make_float2(0.f, 0.f), c2d = make_float2(0.f, 0.f);   // (r, g), (b, depth)
    float2 acc[DP > 0 ? DP / 2 : 1];   // feature channels in packed pairs
#pragma unroll
    for (int c = 0; c < (DP > 0 ? DP / 2 : 1); ++c) acc[c] = make_float2(0.f, 0.f);
    int last = 0;     // 1 + list position of the last blended entry
    int lastk = -1;   // its batch slot, resolved once per batch
    bool done = !it.in_img;
    auto accumulate = [&](int k, float w, float z) {
      const float4 r2 = s_r[3 * k + 2];
      const float2 w2 = splat2(w);
      c01 = fma2(w2, make_float2(r2.x, r2.y), c01);
      c2d = fma2(w2, make_float2(r2.z, z), c2d);
      if constexpr (DP > 0) {
        const float4* f4 = reinterpret_cast<const float4*>(s_f + k * DP);
#pragma unroll
        for (int e = 0; e < DP / 4; ++e) {
          const float4 f = f4[e];
          acc[2 * e] = fma2(w2, make_float2(f.x, f.y), acc[2 * e]);
          acc[2 * e + 1] = fma2(w2, make_float2(f.z, f.w), acc[2 * e + 1]);
        }
      }
    };

    for (int b0 = start; b0 < end; b0 += 32) {
      if (__all_sync(kFull, done)) break;
      const int nk = stage_batch(cam, it, rec, inst_id, b0, end, start, s_r, s_id, s_orig);
      __syncwarp();
      if constexpr (DP > 0) stage_feats<DP, BF16>(feats, D, s_id, nk, s_f);
      __syncwarp();
      int pk = -1;        // entry whose terms are still to be added (software pipeline)
      float pw = 0.f, pz = 0.f;
      bool pany = false;  // some sample of the warp blends it
      for (int k = 0; k < nk; ++k) {
        const float4 r0 = s_r[3 * k];
        const float4 r1 = s_r[3 * k + 1];
        const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
        const float a = fminf(kAlphaMax, __fmul_rn(r1.y, blend_gauss(sigma)));
        // the previous entry is accumulated while this one's opacity is evaluated
        if (pany) accumulate(pk, pw, pz);
        float w = 0.f;
        if (!done && sigma >= 0.f && sigma <= r1.w && a >= kAlphaMin) {
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
          if (Tn < kTMin) {
            done = true;
          } else {
            w = __fmul_rn(a, T);
            T = Tn;
            lastk = k;
          }
        }
        pk = k;
        pw = w;
        pz = r1.z;
        pany = __any_sync(kFull, w != 0.f);
      }
      if (pany) accumulate(pk, pw, pz);   // before the staging slots are refilled
      if (lastk >= 0) { last = s_orig[lastk] + 1; lastk = -1; }
      __syncwarp();   // the staging slots are refilled by the next batch
    }

    const int64_t p = (int64_t)it.m * cam.GW + it.n;
    if (it.in_img) {
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
      T_final[p] = T;
      n_contrib[p] = (uint32_t)last;
    }
    if constexpr (LOSS) {
      // masked L1 + cosine loss of the sample (the same arithmetic as the tile kernel); the
      // target column is parked in the warp's idle feature slots
      if (it.in_img) {
        const float V = fl.mask ? __ldg(fl.mask + p) : 1.f;
        float dot = 0.f, aa = 0.f, bb = 0.f, l1 = 0.f;
#pragma unroll
        for (int c = 0; c < DP; ++c) {
          if (c < D) {
            const float a = V * pair_at(acc, c), b = V * __ldg(fl.target + c * HW + p);
            s_f[c * 32 + lane] = b;
            dot = fmaf(a, b, dot);
            aa = fmaf(a, a, aa);
            bb = fmaf(b, b, bb);
            l1 += fabsf(a - b);
          }
        }
        const float la = sqrtf(aa), lb = sqrtf(bb);
        const float inv = 1.f / (fmaxf(la, kCosEps) * fmaxf(lb, kCosEps));
        const float cosv = dot * inv;
        const float cf = la > kCosEps ? cosv / aa : 0.f;
#pragma unroll
        for (int c = 0; c < DP; ++c) {
          if (c < D) {
            const float a = V * pair_at(acc, c), b = s_f[c * 32 + lane];
            const float sg = a > b ? 1.f : (a < b ? -1.f : 0.f);
            fl.g_feat[c * HW + p] = V * (fl.w_l1 * sg - fl.w_cos * (b * inv - cf * a));
          }
        }
        l1_sum += (double)l1;
        cos_sum += (double)(1.f - cosv);
      }
      __syncwarp();
    }
  }
  if ((threadIdx.x & 31) == 0) queue_leave(tq, gridDim.x * (blockDim.x >> 5));
  if constexpr (LOSS) {
    __shared__ double s_red[2][kWarps];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l1_sum += __shfl_xor_sync(kFull, l1_sum, o);
      cos_sum += __shfl_xor_sync(kFull, cos_sum, o);
    }
    if (lane == 0) {
      s_red[0][warp] = l1_sum;
      s_red[1][warp] = cos_sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kWarps; ++w) {
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

// Samples of the compact grid whose pixel lies outside the image: nothing is rendered
// there (alpha 0, T = 1); with the fused loss their terms (G_hat = 0) are added too.
template <bool LOSS>
__global__ void __launch_bounds__(kGT)
k_grid_fill(CamDev cam, int D, float* __restrict__ rgb, float* __restrict__ depth,
            float* __restrict__ alpha, float* __restrict__ feat, float* __restrict__ T_final,
            uint32_t* __restrict__ n_contrib, FeatLoss fl) {
  const int64_t HW = (int64_t)cam.GW * cam.GH;
  double l1_sum = 0.0, cos_sum = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kGT + threadIdx.x; p < HW; p += (int64_t)gridDim.x * kGT) {
    const int m = (int)(p / cam.GW), n = (int)(p - (int64_t)m * cam.GW);
    if (grid_coord(cam.ox, cam.stride, n) < cam.W && grid_coord(cam.oy, cam.stride, m) < cam.H)
      continue;
    if (rgb) rgb[p] = rgb[HW + p] = rgb[2 * HW + p] = 0.f;
    if (depth) depth[p] = 0.f;
    if (alpha) alpha[p] = 0.f;
    if (feat)
      for (int c = 0; c < D; ++c) feat[c * HW + p] = 0.f;
    T_final[p] = 1.f;
    n_contrib[p] = 0u;
    if constexpr (LOSS) {
      const float V = fl.mask ? __ldg(fl.mask + p) : 1.f;
      float bb = 0.f, l1 = 0.f;
      for (int c = 0; c < D; ++c) {
        const float b = V * __ldg(fl.target + c * HW + p);
        bb = fmaf(b, b, bb);
        l1 += fabsf(b);
      }
      const float inv = 1.f / (kCosEps * fmaxf(sqrtf(bb), kCosEps));
      for (int c = 0; c < D; ++c) {
        const float b = V * __ldg(fl.target + c * HW + p);
        const float sg = b > 0.f ? -1.f : (b < 0.f ? 1.f : 0.f);
        fl.g_feat[c * HW + p] = V * (fl.w_l1 * sg - fl.w_cos * (b * inv));
      }
      l1_sum += (double)l1;
      cos_sum += 1.0;
    }
  }
  if constexpr (LOSS) {
    __shared__ double s_red[2][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l1_sum += __shfl_xor_sync(kFull, l1_sum, o);
      cos_sum += __shfl_xor_sync(kFull, cos_sum, o);
    }
    if (lane == 0) {
      s_red[0][warp] = l1_sum;
      s_red[1][warp] = cos_sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kWarps; ++w) {
        a += s_red[0][w];
        b += s_red[1][w];
      }
      if (a != 0.0 || b != 0.0) {
        a *= fl.s_l1;
        b *= fl.s_cos;
        atomicAdd(fl.loss, fl.lambda * (a + b));
        atomicAdd(fl.loss + 1, a);
        atomicAdd(fl.loss + 2, b);
      }
    }
  }
}

__device__ __forceinline__ void red_add4(float* dst, float a, float b, float c, float d) {
  atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a, b, c, d));
}

template <int DP, bool FO>
constexpr int bwd_warp_floats() {
  // records, ids, list positions, features (not when FO), g_F rows, weights
  return 32 * 12 + 32 + 32 + (FO ? 0 : 32 * DP) + 32 * DP + 32 * kWT;
}

template <int DP, bool BF16, bool FO>
__global__ void __launch_bounds__(kGT, 2)
k_grid_bwd(CamDev cam, TileQueue tq, int CH, const GaussRec* __restrict__ rec,
           const void* __restrict__ feats, int D, const uint2* __restrict__ ranges,
           const uint32_t* __restrict__ inst_id, const float* __restrict__ T_final,
           const uint32_t* __restrict__ n_contrib, const float* __restrict__ g_rgb,
           const float* __restrict__ g_depth, const float* __restrict__ g_alpha,
           const float* __restrict__ g_feat, float* __restrict__ g2d, float* __restrict__ g_feats) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* base = smem + warp * bwd_warp_floats<DP, FO>();
  float4* s_r = reinterpret_cast<float4*>(base);
  uint32_t* s_id = reinterpret_cast<uint32_t*>(base + 32 * 12);
  int* s_orig = reinterpret_cast<int*>(base + 32 * 12 + 32);
  float* s_f = base + 32 * 12 + 64;                    // [32][DP] (not when FO)
  float* s_E = s_f + (FO ? 0 : 32 * DP);               // [32][DP]: g_F of each lane's sample
  float* s_W = s_E + 32 * DP;                          // [32 lanes][kWT]: w per entry
  const int64_t HW = (int64_t)cam.GW * cam.GH;
  constexpr int CB = DP / 4;

  for (;;) {
    const uint32_t q = next_item(tq.head);
    if (q >= (uint32_t)tq.n_tiles) break;
    ItemLane it;
    if (!decode_item(cam, tq, CH, q, &it)) continue;
    const float fx = (float)it.px + 0.5f, fy = (float)it.py + 0.5f;
    const int64_t p = (int64_t)it.m * cam.GW + it.n;
    const uint2 rg = ranges[it.tile];
    const int start = (int)rg.x;

    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f, Tf = 1.f;
    int nc = 0;
    float gF[DP > 0 ? DP : 1];
#pragma unroll
    for (int c = 0; c < (DP > 0 ? DP : 1); ++c) gF[c] = 0.f;
    if (it.in_img) {
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
        for (int c = 0; c < DP; ++c) gF[c] = c < D ? g_feat[c * HW + p] : 0.f;
      }
    }
    if constexpr (DP > 0) {
#pragma unroll
      for (int c = 0; c < DP; c += 4)
        *reinterpret_cast<float4*>(s_E + lane * DP + c) = make_float4(gF[c], gF[c + 1], gF[c + 2], gF[c + 3]);
    }
    int maxn = nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(kFull, maxn, o));
    if (rg.x + (uint32_t)maxn > rg.y) maxn = 0;   // never, for consistent inputs

    float T = Tf, s_run = 0.f;
    const float gAT = gA * Tf;
    for (int c1 = maxn; c1 > 0; c1 -= 32) {
      const int c0 = max(0, c1 - 32);
      const int nk = stage_batch(cam, it, rec, inst_id, start + c0, start + c1, start, s_r, s_id, s_orig);
      __syncwarp();
      if constexpr (DP > 0 && !FO) stage_feats<DP, BF16>(feats, D, s_id, nk, s_f);
      __syncwarp();
      unsigned wlive = 0u;   // entries with a non-zero weight at some sample
      for (int k = nk - 1; k >= 0; --k) {
        float w = 0.f, gs = 0.f, go = 0.f;
        const float4 r0 = s_r[3 * k];
        const float4 r1 = s_r[3 * k + 1];
        // g.x_i does not depend on the blend decisions: formed first, so that it overlaps
        // the opacity evaluation, which is branch-free (the decision selects the updates)
        float dot = 0.f;
        if constexpr (!FO) {
          const float4 r2 = s_r[3 * k + 2];
          float2 d01 = mul2(make_float2(gC0, gC1), make_float2(r2.x, r2.y));
          float2 d23 = mul2(make_float2(gC2, gD), make_float2(r2.z, r1.z));
          if constexpr (DP > 0) {
            const float4* f4 = reinterpret_cast<const float4*>(s_f + k * DP);
#pragma unroll
            for (int e = 0; e < DP / 4; ++e) {
              const float4 f = f4[e];
              d01 = fma2(make_float2(gF[4 * e], gF[4 * e + 1]), make_float2(f.x, f.y), d01);
              d23 = fma2(make_float2(gF[4 * e + 2], gF[4 * e + 3]), make_float2(f.z, f.w), d23);
            }
          }
          dot = (d01.x + d01.y) + (d23.x + d23.y);
        }
        const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
        const float G = blend_gauss(sigma);
        const float oG = __fmul_rn(r1.y, G);
        const float a = fminf(kAlphaMax, oG);
        const bool ok = it.in_img & (s_orig[k] < nc) & (sigma >= 0.f) & (sigma <= r1.w) & (a >= kAlphaMin);
        const float inv = __fdividef(1.f, 1.f - a);
        const float Tn = T * inv;   // T_i
        if (ok) w = a * Tn;
        if constexpr (!FO) {
          const float galpha = Tn * (dot - s_run) + gAT * inv;
          const float sn = a * dot + (1.f - a) * s_run;
          if (ok && oG <= kAlphaMax) {
            go = galpha * G;
            gs = -galpha * a;
          }
          if (ok) s_run = sn;
        }
        if (ok) T = Tn;
        s_W[w_slot(lane, k)] = w;
        const bool any = __any_sync(kFull, w != 0.f);
        if (any) wlive |= 1u << k;
        if constexpr (!FO) {
          if (any) {
            // this Gaussian's terms summed over the item's samples
            const float dx = fx - r0.x, dy = fy - r0.y;
            const float A = r0.z, Bq = r0.w, C = r1.x;
            float v[10] = {-gs * (A * dx + Bq * dy), -gs * (Bq * dx + C * dy), 0.5f * gs * dx * dx,
                           gs * dx * dy,            0.5f * gs * dy * dy,      go,
                           w * gC0,                 w * gC1,                  w * gC2,
                           w * gD};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
              for (int e = 0; e < 10; ++e) v[e] += __shfl_xor_sync(kFull, v[e], o);
            if (lane == 0) {
              float* dst = g2d + (int64_t)s_id[k] * kG2D;
              red_add4(dst, v[0], v[1], v[2], v[3]);
              red_add4(dst + 4, v[4], v[5], v[6], v[7]);
              red_add4(dst + 8, v[8], v[9], 0.f, 0.f);
            }
          }
        }
      }
      __syncwarp();
      // feature gradients of the batch: out[k][c] = sum over the samples of w g_F
      if constexpr (DP > 0) {
        if (g_feats) {
          // 4 entries x 4 channels per task: one 16-byte weight load and one 16-byte g_F
          // load per sample feed 16 FMAs.  Weights of entries >= nk are stale, but only
          // entries with a wlive bit (all < nk) are written out.
          const int nkb = (nk + 3) >> 2;
          for (int task = lane; task < nkb * CB; task += 32) {
            const int kb = task / CB, cb = task - kb * CB, k0 = 4 * kb;
            const unsigned live4 = (wlive >> k0) & 15u;
            if (!live4) continue;
            float2 o[4][2];   // entries x, channels in packed pairs
#pragma unroll
            for (int x = 0; x < 4; ++x) o[x][0] = o[x][1] = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
              const float4 w4 = *reinterpret_cast<const float4*>(s_W + w_slot(l, k0));
              const float4 e = *reinterpret_cast<const float4*>(s_E + l * DP + 4 * cb);
              const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
              for (int x = 0; x < 4; ++x) {
                const float2 w2 = splat2(wv[x]);
                o[x][0] = fma2(w2, make_float2(e.x, e.y), o[x][0]);
                o[x][1] = fma2(w2, make_float2(e.z, e.w), o[x][1]);
              }
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              if (!(live4 >> x & 1u)) continue;
              float* dst = g_feats + (int64_t)s_id[k0 + x] * D + 4 * cb;
              if (D == DP) {
                atomicAdd(reinterpret_cast<float4*>(dst), make_float4(o[x][0].x, o[x][0].y, o[x][1].x, o[x][1].y));
              } else {
#pragma unroll
                for (int y = 0; y < 4; ++y)
                  if (4 * cb + y < D) atomicAdd(dst + y, pair_at(o[x], y));
              }
            }
          }
        }
      }
      __syncwarp();   // the staging slots are refilled by the next batch
    }
  }
}

// Pair counts of a grid render (statistics): one thread per sample walks its tile's list.
__global__ void __launch_bounds__(kGT)
k_grid_pair_stats(CamDev cam, int CH, const GaussRec* __restrict__ rec,
                  const uint2* __restrict__ ranges, const uint32_t* __restrict__ inst_id,
                  const uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ item_max,
                  unsigned long long* __restrict__ stats64) {
  const int64_t HW = (int64_t)cam.GW * cam.GH;
  unsigned long long eval = 0, blend = 0;
  for (int64_t p = (int64_t)blockIdx.x * kGT + threadIdx.x; p < HW; p += (int64_t)gridDim.x * kGT) {
    const int m = (int)(p / cam.GW), n = (int)(p - (int64_t)m * cam.GW);
    const int px = grid_coord(cam.ox, cam.stride, n), py = grid_coord(cam.oy, cam.stride, m);
    if (px >= cam.W || py >= cam.H) continue;
    const int tx = px >> 4, ty = py >> 4, tile = ty * cam.TX + tx;
    const TileSamples ts = tile_samples(cam, tx, ty);
    const int k = (m - ts.m0) * (ts.n1 - ts.n0) + (n - ts.n0);
    const uint32_t nc = n_contrib[p];
    atomicMax(&item_max[(int64_t)tile * CH + k / 32], nc);
    const uint2 rg = ranges[tile];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    for (uint32_t j = 0; j < nc && rg.x + j < rg.y; ++j) {
      const uint32_t id = inst_id[rg.x + j];
      if (id >= (uint32_t)cam.n_gauss) continue;
      const float4 r0 = rec[id].r0, r1 = rec[id].r1;
      ++eval;
      const float sigma = blend_sigma(__fsub_rn(fx, r0.x), __fsub_rn(fy, r0.y), r0.z, r0.w, r1.x);
      if (sigma >= 0.f && fminf(kAlphaMax, __fmul_rn(r1.y, blend_gauss(sigma))) >= kAlphaMin) ++blend;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    eval += __shfl_xor_sync(kFull, eval, o);
    blend += __shfl_xor_sync(kFull, blend, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&stats64[0], eval);
    atomicAdd(&stats64[1], blend);
  }
}

__global__ void __launch_bounds__(kGT)
k_sum_items(const uint32_t* __restrict__ item_max, int64_t n_items, uint32_t* __restrict__ counters) {
  uint32_t s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kGT + threadIdx.x; i < n_items; i += (int64_t)gridDim.x * kGT)
    s += item_max[i];
  s = __reduce_add_sync(kFull, s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(&counters[kCntInstEff], s);
}

int sms_on_device() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

bool has_outside_samples(const CamDev& cam) {
  return grid_coord(cam.ox, cam.stride, cam.GW - 1) >= cam.W ||
         grid_coord(cam.oy, cam.stride, cam.GH - 1) >= cam.H;
}

template <int DP, bool BF16, bool LOSS>
void launch_fwd_t(const CamDev& cam, const TileQueue& tq, int CH, const GaussRec* rec,
                  const void* feats, int D, const uint2* ranges, const uint32_t* inst_id, float* rgb,
                  float* depth, float* alpha, float* feat, float* T_final, uint32_t* n_contrib,
                  const FeatLoss& fl, cudaStream_t st) {
  const size_t smem = sizeof(float) * kWarps * fwd_warp_floats<DP>();
  auto kern = k_grid_fwd<DP, BF16, LOSS>;
  const int grid = persistent_grid(kern, kGT, smem, (int)ceil_div(tq.n_tiles, kWarps));
  kern<<<grid, kGT, smem, st>>>(cam, tq, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha, feat,
                                T_final, n_contrib, fl);
  note_launch();
}

template <int DP>
void launch_fwd_dp(bool bf, bool loss, const CamDev& cam, const TileQueue& tq, int CH,
                   const GaussRec* rec, const void* feats, int D, const uint2* ranges,
                   const uint32_t* inst_id, float* rgb, float* depth, float* alpha, float* feat,
                   float* T_final, uint32_t* n_contrib, const FeatLoss& fl, cudaStream_t st) {
  if constexpr (DP > 0) {
    if (loss) {
      if (bf)
        launch_fwd_t<DP, true, true>(cam, tq, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha,
                                     feat, T_final, n_contrib, fl, st);
      else
        launch_fwd_t<DP, false, true>(cam, tq, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha,
                                      feat, T_final, n_contrib, fl, st);
      return;
    }
  }
  if (bf)
    launch_fwd_t<DP, true, false>(cam, tq, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha,
                                  feat, T_final, n_contrib, fl, st);
  else
    launch_fwd_t<DP, false, false>(cam, tq, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha,
                                   feat, T_final, n_contrib, fl, st);
}

template <int DP, bool BF16, bool FO>
void launch_bwd_t(const CamDev& cam, const TileQueue& tq, int CH, const GaussRec* rec,
                  const void* feats, int D, const uint2* ranges, const uint32_t* inst_id,
                  const float* T_final, const uint32_t* n_contrib, const float* g_rgb,
                  const float* g_depth, const float* g_alpha, const float* g_feat, float* g2d,
                  float* g_feats, cudaStream_t st) {
  const size_t smem = sizeof(float) * kWarps * bwd_warp_floats<DP, FO>();
  auto kern = k_grid_bwd<DP, BF16, FO>;
  const int grid = persistent_grid(kern, kGT, smem, (int)ceil_div(tq.n_tiles, kWarps));
  kern<<<grid, kGT, smem, st>>>(cam, tq, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib,
                                g_rgb, g_depth, g_alpha, g_feat, g2d, g_feats);
  note_launch();
}

template <int DP>
void launch_bwd_dp(bool bf, bool fo, const CamDev& cam, const TileQueue& tq, int CH,
                   const GaussRec* rec, const void* feats, int D, const uint2* ranges,
                   const uint32_t* inst_id, const float* T_final, const uint32_t* n_contrib,
                   const float* g_rgb, const float* g_depth, const float* g_alpha,
                   const float* g_feat, float* g2d, float* g_feats, cudaStream_t st) {
  if constexpr (DP > 0) {
    if (fo) {
      if (bf)
        launch_bwd_t<DP, true, true>(cam, tq, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib,
                                     g_rgb, g_depth, g_alpha, g_feat, g2d, g_feats, st);
      else
        launch_bwd_t<DP, false, true>(cam, tq, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib,
                                      g_rgb, g_depth, g_alpha, g_feat, g2d, g_feats, st);
      return;
    }
  }
  if (bf)
    launch_bwd_t<DP, true, false>(cam, tq, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib,
                                  g_rgb, g_depth, g_alpha, g_feat, g2d, g_feats, st);
  else
    launch_bwd_t<DP, false, false>(cam, tq, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib,
                                   g_rgb, g_depth, g_alpha, g_feat, g2d, g_feats, st);
}

}  // namespace

int grid_chunks_per_tile(int stride) {
  const int per_axis = (16 + stride - 1) / stride;
  return (per_axis * per_axis + 31) / 32;
}

void launch_grid_fwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec, const void* feats,
                     int feat_dtype, int D, const uint2* ranges, const uint32_t* inst_id, float* rgb,
                     float* depth, float* alpha, float* feat, float* T_final, uint32_t* n_contrib,
                     const FeatLoss* loss, cudaStream_t st) {
  if (cam.GW <= 0 || cam.GH <= 0) return;
  const bool bf = feat_dtype == GS_BF16;
  FeatLoss fl{};
  if (loss && D > 0) fl = *loss;
  const bool loss_on = fl.target != nullptr;
  const int CH = grid_chunks_per_tile(cam.stride);
  TileQueue q = tq;
  q.n_tiles = tq.n_tiles * CH;   // work items
  if (tq.n_tiles > 0) {
    const int DP = (feat || loss_on) ? padded_feat(D) : 0;
#define GS_GFWD(dp)                                                                              \
  launch_fwd_dp<dp>(bf, loss_on, cam, q, CH, rec, feats, D, ranges, inst_id, rgb, depth, alpha, \
                    feat, T_final, n_contrib, fl, st)
    switch (DP) {
      case 0: GS_GFWD(0); break;
      case 8: GS_GFWD(8); break;
      case 16: GS_GFWD(16); break;
      case 32: GS_GFWD(32); break;
      default: GS_GFWD(64); break;
    }
#undef GS_GFWD
  }
  if (has_outside_samples(cam)) {
    const int64_t HW = (int64_t)cam.GW * cam.GH;
    const int grid = (int)min64(ceil_div(HW, kGT), (int64_t)sms_on_device() * 8);
    float* fo = (feat && D > 0) ? feat : nullptr;
    if (loss_on)
      k_grid_fill<true><<<grid, kGT, 0, st>>>(cam, D, rgb, depth, alpha, fo, T_final, n_contrib, fl);
    else
      k_grid_fill<false><<<grid, kGT, 0, st>>>(cam, D, rgb, depth, alpha, fo, T_final, n_contrib, fl);
    note_launch();
  }
}

void launch_grid_bwd(const CamDev& cam, const TileQueue& tq, const GaussRec* rec, const void* feats,
                     int feat_dtype, int D, const uint2* ranges, const uint32_t* inst_id,
                     const float* T_final, const uint32_t* n_contrib, const float* g_rgb,
                     const float* g_depth, const float* g_alpha, const float* g_feat, float* g2d,
                     float* g_feats, bool features_only, cudaStream_t st) {
  if (cam.GW <= 0 || cam.GH <= 0 || tq.n_tiles <= 0) return;
  const bool bf = feat_dtype == GS_BF16;
  const int DP = g_feat ? padded_feat(D) : 0;
  const bool fo = features_only && DP > 0 && g_feats;
  const int CH = grid_chunks_per_tile(cam.stride);
  TileQueue q = tq;
  q.n_tiles = tq.n_tiles * CH;
#define GS_GBWD(dp)                                                                              \
  launch_bwd_dp<dp>(bf, fo, cam, q, CH, rec, feats, D, ranges, inst_id, T_final, n_contrib, g_rgb, \
                    g_depth, g_alpha, g_feat, g2d, g_feats, st)
  switch (DP) {
    case 0: GS_GBWD(0); break;
    case 8: GS_GBWD(8); break;
    case 16: GS_GBWD(16); break;
    case 32: GS_GBWD(32); break;
    default: GS_GBWD(64); break;
  }
#undef GS_GBWD
}

void launch_grid_stats(const CamDev& cam, const GaussRec* rec, const uint2* ranges,
                       const uint32_t* inst_id, const uint32_t* n_contrib, uint32_t* item_max,
                       uint32_t* counters, unsigned long long* stats64, cudaStream_t st) {
  const int CH = grid_chunks_per_tile(cam.stride);
  const int64_t n_items = (int64_t)cam.TX * cam.TY * CH;
  cudaMemsetAsync(stats64, 0, 2 * sizeof(unsigned long long), st);
  cudaMemsetAsync(counters + kCntInstEff, 0, sizeof(uint32_t), st);
  if (n_items <= 0 || cam.GW <= 0 || cam.GH <= 0) return;
  cudaMemsetAsync(item_max, 0, sizeof(uint32_t) * (size_t)n_items, st);
  const int64_t HW = (int64_t)cam.GW * cam.GH;
  const int grid = (int)min64(ceil_div(HW, kGT), (int64_t)sms_on_device() * 8);
  k_grid_pair_stats<<<grid, kGT, 0, st>>>(cam, CH, rec, ranges, inst_id, n_contrib, item_max, stats64);
  const int g2 = (int)min64(ceil_div(n_items, kGT), (int64_t)sms_on_device() * 4);
  k_sum_items<<<g2, kGT, 0, st>>>(item_max, n_items, counters);
  note_launch(2);
}

}  // namespace gs
