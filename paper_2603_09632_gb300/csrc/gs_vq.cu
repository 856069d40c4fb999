// VQ semantic parameterisation (X-GS Sec. 3.2 "Online VQ Module") and the per-pixel decode
// of App. E: each Gaussian carries logits z_i over a shared codebook E [L x D]; the renderer
// splats the mixture weights w_i = softmax(z_i) (the feature path with n_feat = L), and a
// pixel's semantic feature is F(x) = E^T w(x).  Prompt relevance (App. E):
// R(x | p) = max_n softmax(tau [F~.t+, F~.t_n-])_1 with F~ = F / (|F| + eps).
//
// The decode is the one dense contraction of the path: [P x L] x [L x D] per frame (at
// 1200x680 with L = 64, D = 512: 53 GFLOP, 1.67 GB of fp32 output), so it runs on the
// 5th-generation tensor cores: tcgen05.mma (kind::tf32, fp32 accumulate in tensor memory)
// issued by one thread per CTA on 128-pixel tiles, operands staged in shared memory in the
// canonical K-major core-matrix layout, completion signalled through an mbarrier, and the
// epilogue (optional F write, |F|^2, relevance) reading the accumulator with tcgen05.ld.
// The next tile's weights are fetched while the tensor cores and the epilogue run.  One
// persistent CTA per SM holds the codebook in shared memory for its range of tiles.  Every
// wait is bounded; on a timeout the kernel records an error, waits (bounded) for its own
// MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kVT = 512;             // threads per CTA (four per tile row)
constexpr int kGroups = kVT / 128;   // threads per row = column groups of the epilogue
constexpr int kRows = 128;           // tile rows (pixels) = TMEM lanes = MMA M
constexpr int kMaxL = 64;            // K
constexpr int kMaxDc = 512;          // N (two MMAs of N = 256)
constexpr int kMaxText = 8;                 // prompt + negatives (read as two float4 per codeword)
constexpr uint32_t kWaitLimit = 1u << 20;   // try_wait polls (each may suspend briefly)
constexpr int kMaxResident = 2048 / kVT;   // CTAs per SM allowed by the thread count

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Canonical K-major, no-swizzle layout: 8-row x 16-byte core matrices; the matrix element
// (row r, k) of a [rows x K] fp32 operand lives at
//   (r / 8) * SBO + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4   bytes,  SBO = (K / 4) * 128.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;          // descriptor version for tcgen05
  // base offset 0, absolute LBO mode 0, layout type 0 = no swizzle
  return d;
}

// Instruction descriptor of kind::tf32: fp32 accumulator, tf32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                       // D format: f32
         | (2u << 7)                     // A format: tf32
         | (2u << 10)                    // B format: tf32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

struct DecodeArgs {
  const float* wmap;      // [L][P]
  int64_t P;
  int L;
  const float* E;         // [L][Dc]
  int Dc;
  float* F;               // [Dc][P] or null
  const float* text;      // [n_text][Dc] or null
  int n_text;
  float tau, eps;
  float* rel;             // [P] or null
  int32_t* err;           // set to 1 on a timed-out wait
};

// Shared-memory plan of the decode CTA (bytes).  The prompt embeddings are staged in the
// partial-dot area, which is only used once the tiles start.
struct DecodeSmem {
  uint32_t a, b, et, dot, nrm, text, bar, tmem, total;
  __host__ __device__ DecodeSmem(int L, int Dc) {
    a = 0;                                              // A tile [128 x L] fp32, core layout
    b = a + (uint32_t)kRows * L * 4;                    // B = E^T [Dc x L] fp32, core layout
    et = b + (uint32_t)Dc * L * 4;                      // E t_j  [L][kMaxText]
    dot = et + (uint32_t)kMaxL * kMaxText * 4;          // [2 buffers][groups][kMaxText][128]
    text = dot;                                         // prompt embeddings [kMaxText][Dc]
    nrm = dot + 2u * kGroups * kMaxText * kRows * 4;    // [2 buffers][groups][128]
    bar = nrm + 2u * kGroups * kRows * 4;
    tmem = bar + 8;
    total = tmem + 8;
  }
};
static_assert(2 * kGroups * kMaxText * kRows >= kMaxText * kMaxDc, "text staging must fit");
static_assert(kMaxText == 8, "E t_j rows are read as two float4");

// One 128-pixel tile per iteration.  The four threads t = r + 128 g (g = 0..3) share row r
// (pixel p = tile * 128 + r): each loads a quarter of the row's L weights (issued before
// the previous tile's epilogue and consumed after it), and in the epilogue warp w reads TMEM lanes 32 (w mod 4) ..
// and every fourth 32-column chunk of F starting at chunk w / 4.  The prompt dot products
// use F.t_j = w.(E t_j) with E t_j formed once per CTA, so the epilogue only adds |F|^2.
__global__ void __launch_bounds__(kVT, 1) k_vq_decode(DecodeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int r = t & (kRows - 1), h = t >> 7;   // row, column group
  const int L = a.L, Dc = a.Dc, LH = L / kGroups;   // weights per thread (L multiple of 8)
  const bool want_rel = a.rel != nullptr;
  const DecodeSmem sm(L, Dc);
  float* sA = reinterpret_cast<float*>(smem + sm.a);
  float* sB = reinterpret_cast<float*>(smem + sm.b);
  float* sEt = reinterpret_cast<float*>(smem + sm.et);
  float* sDot = reinterpret_cast<float*>(smem + sm.dot);
  float* sNrm = reinterpret_cast<float*>(smem + sm.nrm);
  float* sTx = reinterpret_cast<float*>(smem + sm.text);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + sm.bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + sm.tmem);
  const uint32_t sbo = (uint32_t)(L / 4) * 128u;   // bytes between 8-row groups

  int ncols = 32;
  while (ncols < Dc) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // codebook, transposed into the K-major B operand: element (n, k) = E[k][n]
  for (int e = t; e < L * Dc; e += kVT) {
    const int k = e / Dc, n = e - k * Dc;
    const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 2) * 128u + (uint32_t)(n & 7) * 16u +
                         (uint32_t)(k & 3) * 4u;
    *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sB) + off) = __ldg(a.E + e);
  }
  const int nt = want_rel ? a.n_text : 0;
  for (int e = t; e < nt * Dc; e += kVT) sTx[e] = __ldg(a.text + e);
  __syncthreads();
  // E t_j for every codeword k (one warp per codeword row, lanes over the D columns)
  for (int k = warp; k < L && nt > 0; k += kVT / 32) {
    float acc[kMaxText];
#pragma unroll
    for (int j = 0; j < kMaxText; ++j) acc[j] = 0.f;
    for (int c = lane; c < Dc; c += 32) {
      const float ev = __ldg(a.E + (int64_t)k * Dc + c);
#pragma unroll
      for (int j = 0; j < kMaxText; ++j)
        if (j < nt) acc[j] = fmaf(ev, sTx[j * Dc + c], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kMaxText; ++j) {
      float v = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sEt[k * kMaxText + j] = v;
    }
  }
  __syncthreads();

  const uint32_t tmem = *s_tmem;
  const uint32_t bar = smem_u32(s_bar);
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
  const int64_t n_tiles = (a.P + kRows - 1) / kRows;

  // this thread's quarter row of weights for one tile (load_rows), and its partial prompt
  // dot products (row_dots, formed when the row is staged)
  float wv[kMaxL / kGroups];
  float dp[kMaxText];
  auto load_rows = [&](int64_t tile) {
    const int64_t p = tile * kRows + r;
    const bool live = p < a.P;
#pragma unroll
    for (int k = 0; k < kMaxL / kGroups; ++k)
      wv[k] = (k < LH && live) ? __ldg(a.wmap + (int64_t)(h * LH + k) * a.P + p) : 0.f;
  };
  auto row_dots = [&]() {
#pragma unroll
    for (int j = 0; j < kMaxText; ++j) dp[j] = 0.f;
    if (nt > 0) {
      // E t_j of codeword k: two 16-byte loads for the kMaxText = 8 prompts
      const float4* et4 = reinterpret_cast<const float4*>(sEt);
#pragma unroll
      for (int k = 0; k < kMaxL / kGroups; ++k) {
        if (k < LH) {
          const float4 e0 = et4[(h * LH + k) * 2], e1 = et4[(h * LH + k) * 2 + 1];
          dp[0] = fmaf(wv[k], e0.x, dp[0]);
          dp[1] = fmaf(wv[k], e0.y, dp[1]);
          dp[2] = fmaf(wv[k], e0.z, dp[2]);
          dp[3] = fmaf(wv[k], e0.w, dp[3]);
          dp[4] = fmaf(wv[k], e1.x, dp[4]);
          dp[5] = fmaf(wv[k], e1.y, dp[5]);
          dp[6] = fmaf(wv[k], e1.z, dp[6]);
          dp[7] = fmaf(wv[k], e1.w, dp[7]);
        }
      }
    }
  };
  auto store_rows = [&](int buf) {
    // a thread's LH = L / 4 weights fill whole 4-element core-matrix rows when LH is a
    // multiple of 4 (L = 16, 32, 48, 64); otherwise (L = 8, 24, 40, 56) store scalars
    if (LH % 4 == 0) {
#pragma unroll
      for (int q = 0; q < kMaxL / kGroups / 4; ++q) {
        if (q < LH / 4) {
          const uint32_t off = (uint32_t)(r >> 3) * sbo + (uint32_t)(h * LH / 4 + q) * 128u + (uint32_t)(r & 7) * 16u;
          *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(sA) + off) =
              make_float4(wv[4 * q], wv[4 * q + 1], wv[4 * q + 2], wv[4 * q + 3]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMaxL / kGroups; ++k) {
        if (k < LH) {
          const int kk = h * LH + k;
          const uint32_t off = (uint32_t)(r >> 3) * sbo + (uint32_t)(kk >> 2) * 128u + (uint32_t)(r & 7) * 16u +
                               (uint32_t)(kk & 3) * 4u;
          *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sA) + off) = wv[k];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxText; ++j)
      if (j < nt) sDot[((buf * kGroups + h) * kMaxText + j) * kRows + r] = dp[j];
  };

  // relevance of a finished tile from its partial norms and prompt dots (buffer it & 1);
  // run one tile later, while the next tile's MMAs and the other warps' stores proceed
  auto finish_rel = [&](int64_t tl, int itl) {
    const int64_t pr = tl * kRows + r;
    if (pr >= a.P) return;
    const int buf = itl & 1;
    float nrm = 0.f;
    for (int g = 0; g < kGroups; ++g) nrm += sNrm[(buf * kGroups + g) * kRows + r];
    const float inv = 1.f / (sqrtf(nrm) + a.eps);
    float d[kMaxText];
#pragma unroll
    for (int j = 0; j < kMaxText; ++j) {
      d[j] = 0.f;
      if (j < nt)
        for (int g = 0; g < kGroups; ++g) d[j] += sDot[((buf * kGroups + g) * kMaxText + j) * kRows + r];
    }
    float best = 0.f;
#pragma unroll
    for (int j = 1; j < kMaxText; ++j)
      if (j < nt) best = fmaxf(best, 1.f / (1.f + __expf(a.tau * (d[j] - d[0]) * inv)));
    a.rel[pr] = best;
  };

  // each CTA decodes one contiguous range of tiles
  const int64_t t_per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_begin = min(n_tiles, (int64_t)blockIdx.x * t_per), t_end = min(n_tiles, t_begin + t_per);
  int64_t tile = t_begin;
  if (tile < t_end) {
    load_rows(tile);
    row_dots();
    store_rows(0);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  uint32_t phase = 0;
  bool failed = false;
  for (int it = 0; tile < t_end; ++tile, ++it) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      for (int ks = 0; ks < L / 8; ++ks) {
        const uint64_t ad = smem_desc(a_base + 256u * ks, 128u, sbo);
        for (int n0 = 0; n0 < Dc; n0 += 256) {
          const int N = min(256, Dc - n0);
          const uint64_t bd = smem_desc(b_base + (uint32_t)(n0 >> 3) * sbo + 256u * ks, 128u, sbo);
          mma_tf32(tmem + (uint32_t)n0, ad, bd, idesc_tf32(kRows, N), ks > 0 ? 1u : 0u);
        }
      }
      mma_commit(bar);
    }
    // issue the next tile's weight loads (first used after this tile's epilogue, so their
    // latency hides behind its stores) and finish the previous tile's relevance while the
    // tensor cores run
    const int64_t next = tile + 1;
    if (next < t_end) load_rows(next);
    if (want_rel && h == 0 && it > 0) finish_rel(tile - 1, it - 1);
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {   // every thread takes the same branch
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: TMEM lanes 32 (warp mod 4) .. + 31 = pixels; chunks h, h + 4, ... of F
    const int64_t p = tile * kRows + 32 * (warp & 3) + lane;
    const bool store = p < a.P && a.F != nullptr;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    float n4[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = 32 * h; c0 < Dc; c0 += 32 * kGroups) {
      float v[32];
      tmem_ld32(lane_addr + (uint32_t)c0, v);
      const int nv = min(32, Dc - c0);   // a multiple of 16
      if (store) {
        float* fp = a.F + (int64_t)c0 * a.P + p;
        if (nv == 32) {
#pragma unroll
          for (int j = 0; j < 32; ++j, fp += a.P) *fp = v[j];
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j, fp += a.P) *fp = v[j];
        }
      }
      if (want_rel) {
#pragma unroll
        for (int j = 0; j < 16; ++j) n4[j & 3] = fmaf(v[j], v[j], n4[j & 3]);
        if (nv == 32) {
#pragma unroll
          for (int j = 16; j < 32; ++j) n4[j & 3] = fmaf(v[j], v[j], n4[j & 3]);
        }
      }
    }
    if (want_rel)
      sNrm[((it & 1) * kGroups + h) * kRows + 32 * (warp & 3) + lane] = (n4[0] + n4[1]) + (n4[2] + n4[3]);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // MMA done, TMEM read, previous relevance done: A and the other buffers free
    if (next < t_end) {
      row_dots();
      store_rows((it + 1) & 1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // next A tile staged; norms and dots consumed
  }
  if (failed) {
    if (t == 0 && a.err) atomicExch(a.err, 1);
    mbar_wait(bar, phase ^ 1u);   // bounded: let this CTA's own MMAs drain before freeing TMEM
  } else if (want_rel && h == 0 && t_begin < t_end) {
    // the last tile's relevance (its partials were published by the loop's last barrier)
    const int64_t last = t_end - 1;
    finish_rel(last, (int)(last - t_begin));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

// w_i = softmax(z_i): one warp per Gaussian, L <= 64 logits (two per lane).
template <bool BF16>
__global__ void __launch_bounds__(256)
k_vq_weights(const float* __restrict__ z, int64_t n, int L, void* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5;
  if (row >= n) return;
  const float* zr = z + row * L;
  const float a = lane < L ? zr[lane] : -INFINITY, b = lane + 32 < L ? zr[lane + 32] : -INFINITY;
  float m = fmaxf(a, b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float ea = lane < L ? __expf(a - m) : 0.f, eb = lane + 32 < L ? __expf(b - m) : 0.f;
  float s = ea + eb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float inv = 1.f / s;
  if constexpr (BF16) {
    __nv_bfloat16* wr = static_cast<__nv_bfloat16*>(w) + row * L;
    if (lane < L) wr[lane] = __float2bfloat16_rn(ea * inv);
    if (lane + 32 < L) wr[lane + 32] = __float2bfloat16_rn(eb * inv);
  } else {
    float* wr = static_cast<float*>(w) + row * L;
    if (lane < L) wr[lane] = ea * inv;
    if (lane + 32 < L) wr[lane + 32] = eb * inv;
  }
}

// dL/dz_i = w_i * (g_i - sum_l g_il w_il), recomputing w_i from z_i.
__global__ void __launch_bounds__(256)
k_vq_weights_bwd(const float* __restrict__ z, const float* __restrict__ g, int64_t n, int L,
                 float* __restrict__ gz) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5;
  if (row >= n) return;
  const float* zr = z + row * L;
  const float* gr = g + row * L;
  const float a = lane < L ? zr[lane] : -INFINITY, b = lane + 32 < L ? zr[lane + 32] : -INFINITY;
  float m = fmaxf(a, b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float ea = lane < L ? __expf(a - m) : 0.f, eb = lane + 32 < L ? __expf(b - m) : 0.f;
  float s = ea + eb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float wa = ea / s, wb = eb / s;
  const float ga = lane < L ? gr[lane] : 0.f, gb = lane + 32 < L ? gr[lane + 32] : 0.f;
  float d = wa * ga + wb * gb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if (lane < L) gz[row * L + lane] = wa * (ga - d);
  if (lane + 32 < L) gz[row * L + lane + 32] = wb * (gb - d);
}

size_t decode_smem(int L, int Dc) { return DecodeSmem(L, Dc).total; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_vq_weights(const float* logits, int64_t n, int32_t L, int32_t out_dtype, void* w_out,
                        void* stream) {
  if (n < 0 || L <= 0 || L > kMaxL || (out_dtype != GS_F32 && out_dtype != GS_BF16) ||
      (n > 0 && (!logits || !w_out)))
    return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const unsigned grid = (unsigned)ceil_div(n * 32, 256);
  if (out_dtype == GS_BF16)
    k_vq_weights<true><<<grid, 256, 0, (cudaStream_t)stream>>>(logits, n, L, w_out);
  else
    k_vq_weights<false><<<grid, 256, 0, (cudaStream_t)stream>>>(logits, n, L, w_out);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_vq_weights_bwd(const float* logits, const float* g_w, int64_t n, int32_t L,
                            float* g_logits, void* stream) {
  if (n < 0 || L <= 0 || L > kMaxL || (n > 0 && (!logits || !g_w || !g_logits))) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const unsigned grid = (unsigned)ceil_div(n * 32, 256);
  k_vq_weights_bwd<<<grid, 256, 0, (cudaStream_t)stream>>>(logits, g_w, n, L, g_logits);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_vq_decode(const float* wmap, int64_t P, int32_t L, const float* codebook, int32_t Dc,
                       float* F_out, const float* text, int32_t n_text, float tau,
                       float* relevance, int32_t* err, void* stream) {
  if (P < 0 || L < 8 || L > kMaxL || L % 8 != 0 || Dc < 16 || Dc > kMaxDc || Dc % 16 != 0 ||
      (P > 0 && (!wmap || !codebook)) || (relevance && (!text || n_text < 2 || n_text > kMaxText)))
    return GS_ERR_ARG;
  if (P == 0 || (!F_out && !relevance)) return GS_OK;
  int dev = 0, sms = 1, smem_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // At most 512 / ncols CTAs may hold their tensor memory on one SM at a time: request
  // enough shared memory that no more than that many are resident (a further CTA would only
  // wait inside its allocation).
  int ncols = 32;
  while (ncols < Dc) ncols <<= 1;
  const int per_sm = 512 / ncols;
  size_t smem = decode_smem(L, Dc);
  if (per_sm < kMaxResident && smem_sm > 0)
    smem = std::max<size_t>(smem, (size_t)smem_sm / (size_t)(per_sm + 1) + 1024);
  if (cudaFuncSetAttribute(k_vq_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return GS_ERR_CUDA;
  DecodeArgs a{wmap, P, L, codebook, Dc, F_out, text, relevance ? n_text : 0, tau, 1e-8f,
               relevance, err};
  const int64_t n_tiles = (P + kRows - 1) / kRows;
  const unsigned grid = (unsigned)min64(n_tiles, (int64_t)sms * per_sm);
  k_vq_decode<<<grid, kVT, smem, (cudaStream_t)stream>>>(a);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
