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
// Products are FP32-accurate by the 3xTF32 split: each operand x = hi + lo with hi and lo
// rounded to tf32 (|x - hi - lo| <= 2^-22 |x|), and W E = Whi Ehi + Wlo Ehi + Whi Elo (the
// dropped Wlo Elo is below 2^-22 of the product).  The split codebook of D = 512 columns
// does not fit one CTA's shared memory, so above 256 columns a cluster of two CTAs (two
// SMs) decodes the same tiles, each its half of the columns; the second CTA forms the
// prompt dots of the relevance and sends them with its half norms |F|^2 to the first CTA
// through distributed shared memory (st.async completing an mbarrier).  Each CTA
// keeps two accumulators in tensor memory, so the next tile's MMAs run during this tile's
// epilogue, and the next weights are fetched while both run.  Every mbarrier wait is
// bounded; on a timeout the kernel records an error, finishes its part of the pair's
// exchange (bounded waits), meets the pair's final cluster barrier, waits (bounded) for its
// own MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kVT = 512;             // threads per CTA (four per tile row when staging)
constexpr int kGroups = 4;           // threads per row when staging = column groups of the epilogue
constexpr int kRows = 128;           // tile rows (pixels) = TMEM lanes = MMA M
constexpr int kMaxL = 64;            // K
constexpr int kMaxDc = 512;          // D
constexpr int kMaxDh = 256;          // columns of one CTA = N of one MMA
constexpr int kMaxText = 8;                 // prompt + negatives (read as two float4 per codeword)
constexpr int kDotBufs = 3;                 // prompt-dot buffers (staged two tiles ahead of use)
constexpr int kXBufs = 3;                   // norm and exchange buffers (relevance two tiles behind)
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

// x rounded to the nearest tf32 value (10 fraction bits, ties away from zero), as fp32.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The 3xTF32 split: x = hi + lo + r with hi, lo exact in tf32 and |r| <= 2^-22 |x|
// (x - hi is exact in fp32).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctas() {
  uint32_t n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}

// Split cluster barrier: arrive publishes this thread's earlier shared-memory writes
// (release), wait returns once every thread of the cluster has arrived (acquire).  Every
// thread of both CTAs takes part, the same number of times.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local), "r"(rank));
  return ra;
}

// Asynchronous 4-byte store into another CTA's shared memory that completes 4 bytes of the
// transaction count of that CTA's mbarrier rbar (no fence on this thread's other writes).
__device__ __forceinline__ void st_async_f32(uint32_t raddr, float v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr),
               "r"(__float_as_uint(v)), "r"(rbar)
               : "memory");
}

// The one arrival of an mbarrier phase, expecting `bytes` of asynchronous stores.
__device__ __forceinline__ void mbar_arrive_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Arrival on an mbarrier of another CTA of the cluster (a "buffer consumed" signal: the
// reads it follows have completed, their values are in registers or already stored).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t rmbar) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(rmbar) : "memory");
}

// Bounded wait for a phase completed by another CTA of the cluster.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
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
  int Dh0;                // columns of the cluster's first CTA (all Dc without a partner)
  float* F;               // [Dc][P] or null
  const float* text;      // [n_text][Dc] or null
  int n_text;
  float tau, eps;
  float* rel;             // [P] or null
  int32_t* err;           // set to 1 on a timed-out wait
};

// Shared-memory plan of the decode CTA (bytes), for L codewords and at most Dh columns.
struct DecodeSmem {
  uint32_t a_hi, a_lo, b_hi, b_lo, et, dot, nrm, peer, bar, xbar, tmem, total;
  __host__ __device__ DecodeSmem(int L, int Dh) {
    a_hi = 0;                                           // weights [128 x L], tf32 hi part
    a_lo = a_hi + (uint32_t)kRows * L * 4;              // ... and lo part
    b_hi = a_lo + (uint32_t)kRows * L * 4;              // E^T [Dh x L] of this CTA's columns
    b_lo = b_hi + (uint32_t)Dh * L * 4;
    et = b_lo + (uint32_t)Dh * L * 4;                   // E t_j  [L + groups][kMaxText], padded
    dot = et + (uint32_t)(kMaxL + kGroups) * kMaxText * 4;   // prompt dots [kDotBufs][kMaxText][128]
    nrm = dot + (uint32_t)kDotBufs * kMaxText * kRows * 4;   // |F|^2 parts [kXBufs][groups][128]
    peer = nrm + (uint32_t)kXBufs * kGroups * kRows * 4;     // from the partner [kXBufs][1 + kMaxText][128]:
    bar = peer + (uint32_t)kXBufs * (1 + kMaxText) * kRows * 4;   // its |F|^2, the prompt dots; MMA completion
    xbar = bar + 8;                                     // exchange buffer full[kXBufs] (first CTA),
    tmem = xbar + 16 * kXBufs;                          // ... consumed[kXBufs] (second CTA)
    total = tmem + 8;
  }
};
static_assert(kMaxText == 8, "E t_j rows are read as two float4");

// One 128-pixel tile per iteration.  Staging: warp w stages rows 8w .. 8w + 7, lanes r,
// r + 8, r + 16, r + 24 share a row, each loading a quarter of its L weights (issued two
// tiles ahead, consumed after the MMAs of the tile before), splitting them into tf32 hi/lo
// parts and forming its part of the prompt dots F.t_j = w.(E t_j) (E t_j formed once per
// CTA).  Epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (pixels) and every fourth
// 32-column chunk of this CTA's columns starting at chunk w / 4, and writes F channel-major.
__global__ void __launch_bounds__(kVT, 1) k_vq_decode(DecodeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int sr = 8 * warp + (lane & 7), sh = lane >> 3;   // staging row, its quarter
  const int L = a.L, LH = L / kGroups;                   // weights per staging thread
  const uint32_t rank = cluster_rank(), nrank = cluster_ctas();
  const int n_lo = rank == 0 ? 0 : a.Dh0;                // this CTA's columns [n_lo, n_lo + Dh)
  const int Dh = rank == 0 ? a.Dh0 : a.Dc - a.Dh0;
  const int Db = (Dh + 31) & ~31;                        // TMEM columns per accumulator
  const bool want_rel = a.rel != nullptr;
  const bool rel_here = want_rel && rank == 0;           // relevance formed by the first CTA
  const bool exch = want_rel && nrank > 1;               // the partner sends |F|^2 and dots
  const DecodeSmem sm(L, a.Dh0);
  float* sAh = reinterpret_cast<float*>(smem + sm.a_hi);
  float* sAl = reinterpret_cast<float*>(smem + sm.a_lo);
  float* sBh = reinterpret_cast<float*>(smem + sm.b_hi);
  float* sBl = reinterpret_cast<float*>(smem + sm.b_lo);
  float* sEt = reinterpret_cast<float*>(smem + sm.et);
  float* sDot = reinterpret_cast<float*>(smem + sm.dot);
  float* sNrm = reinterpret_cast<float*>(smem + sm.nrm);
  float* sPeer = reinterpret_cast<float*>(smem + sm.peer);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + sm.bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + sm.tmem);
  const uint32_t sbo = (uint32_t)(L / 4) * 128u;   // bytes between 8-row groups

  int ncols = 32;
  while (ncols < 2 * Db) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int k = 0; k < 1 + 2 * kXBufs; ++k)   // MMA completion, full[kXBufs], consumed[kXBufs]
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(smem + sm.bar + 8 * k)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // E t_j for every codeword k over all Dc columns, in the CTA that forms the prompt dots
  // (the second of a pair, or the only one).  The prompts are staged in the operand area,
  // idle until the codebook and the first tile are staged (n_text Dc <= 8 Dc floats fit:
  // the A and B areas hold 2 L (128 + Dh) >= 8 Dc floats for L >= 8 and Dh >= Dc / 2); one
  // warp per codeword, lanes over the columns.
  const int ntx = want_rel ? a.n_text : 0;                 // prompts of the relevance
  const int nt = (want_rel && rank == nrank - 1) ? ntx : 0;  // ... whose dots this CTA forms
  if (nt > 0) {
    float* sTx = sAh;
    for (int e = t; e < nt * a.Dc; e += kVT) sTx[e] = __ldg(a.text + e);
    __syncthreads();
    for (int k = warp; k < L; k += kVT / 32) {
      float acc[kMaxText];
#pragma unroll
      for (int j = 0; j < kMaxText; ++j) acc[j] = 0.f;
#pragma unroll 4
      for (int c = lane; c < a.Dc; c += 32) {
        const float ev = __ldg(a.E + (int64_t)k * a.Dc + c);
#pragma unroll
        for (int j = 0; j < kMaxText; ++j)
          if (j < nt) acc[j] = fmaf(ev, sTx[j * a.Dc + c], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < kMaxText; ++j) {
        float v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sEt[(k + k / LH) * kMaxText + j] = v;
      }
    }
    __syncthreads();   // the operand area is free again
  }
  // this CTA's codebook columns, transposed into the K-major B operand and split:
  // element (n, k) = E[k][n_lo + n]
  for (int e = t; e < L * Dh; e += kVT) {
    const int k = e / Dh, n = e - k * Dh;
    const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 2) * 128u + (uint32_t)(n & 7) * 16u +
                         (uint32_t)(k & 3) * 4u;
    float hi, lo;
    split_tf32(__ldg(a.E + (int64_t)k * a.Dc + n_lo + n), hi, lo);
    *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sBh) + off) = hi;
    *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sBl) + off) = lo;
  }
  __syncthreads();
  // the partner's exchange barriers are initialised before either CTA signals the other
  if (exch) {
    cluster_arrive();
    cluster_wait();
  }

  const uint32_t tmem = *s_tmem;
  const uint32_t bar = smem_u32(s_bar);
  const uint32_t full0 = smem_u32(smem + sm.xbar), cons0 = full0 + 8 * kXBufs;   // + 8 b for buffer b
  // relevance of tile i is finished in iteration i + lag (after the last tile, in the tail):
  // one tile behind in a single CTA, two behind in a pair, so that the partner's data for a
  // tile, sent as it finishes the tile, is normally in before it is needed
  const int lag = exch ? 2 : 1;
  bool xfer_ok = true;   // this thread's exchange waits have not timed out
  const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
  const uint32_t idesc = idesc_tf32(kRows, Dh);
  const int64_t n_tiles = (a.P + kRows - 1) / kRows;

  // this thread's quarter row of weights for one tile
  float wv[kMaxL / kGroups];
  auto load_rows = [&](int64_t tile) {
    const int64_t p = tile * kRows + sr;
    const bool live = p < a.P;
#pragma unroll
    for (int k = 0; k < kMaxL / kGroups; ++k)
      wv[k] = (k < LH && live) ? __ldg(a.wmap + (int64_t)(sh * LH + k) * a.P + p) : 0.f;
  };
  // split the held weights into the A operands
  auto stage_a = [&]() {
    unsigned char* Ah = reinterpret_cast<unsigned char*>(sAh);
    unsigned char* Al = reinterpret_cast<unsigned char*>(sAl);
    const uint32_t row = (uint32_t)warp * sbo + (uint32_t)(sr & 7) * 16u;
    if (LH % 4 == 0) {   // whole 4-element core-matrix rows (L = 16, 32, 48, 64)
#pragma unroll
      for (int q = 0; q < kMaxL / kGroups / 4; ++q) {
        if (q < LH / 4) {
          float4 h4, l4;
          split_tf32(wv[4 * q], h4.x, l4.x);
          split_tf32(wv[4 * q + 1], h4.y, l4.y);
          split_tf32(wv[4 * q + 2], h4.z, l4.z);
          split_tf32(wv[4 * q + 3], h4.w, l4.w);
          const uint32_t off = row + (uint32_t)(sh * LH / 4 + q) * 128u;
          *reinterpret_cast<float4*>(Ah + off) = h4;
          *reinterpret_cast<float4*>(Al + off) = l4;
        }
      }
    } else {             // L = 8, 24, 40, 56: scalars
#pragma unroll
      for (int k = 0; k < kMaxL / kGroups; ++k) {
        if (k < LH) {
          const int kk = sh * LH + k;
          const uint32_t off = row + (uint32_t)(kk >> 2) * 128u + (uint32_t)(kk & 3) * 4u;
          float hi, lo;
          split_tf32(wv[k], hi, lo);
          *reinterpret_cast<float*>(Ah + off) = hi;
          *reinterpret_cast<float*>(Al + off) = lo;
        }
      }
    }
  };
  // the prompt dots of the held row (nt > 0), summed over its four quarters by
  // shuffles and kept in dot buffer dbuf.  E t_j is stored with one padding row per quarter,
  // so the four quarters of a warp read four different bank groups.
  auto stage_dots = [&](int dbuf) {
    if (nt > 0) {
      float dp[kMaxText];
#pragma unroll
      for (int j = 0; j < kMaxText; ++j) dp[j] = 0.f;
      const float4* et4 = reinterpret_cast<const float4*>(sEt);
#pragma unroll
      for (int k = 0; k < kMaxL / kGroups; ++k) {
        if (k < LH) {
          const float4 e0 = et4[(sh * (LH + 1) + k) * 2], e1 = et4[(sh * (LH + 1) + k) * 2 + 1];
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
#pragma unroll
      for (int j = 0; j < kMaxText; ++j) {
        dp[j] += __shfl_xor_sync(0xffffffffu, dp[j], 8);
        dp[j] += __shfl_xor_sync(0xffffffffu, dp[j], 16);
      }
      // quarter sh stores prompts 2 sh and 2 sh + 1 of its row
#pragma unroll
      for (int j = 0; j < kMaxText; ++j)
        if ((j >> 1) == sh) sDot[(dbuf * kMaxText + j) * kRows + sr] = dp[j];
    }
  };
  // 3 L/8 MMAs of M = 128, N = Dh, K = 8 into accumulator buf (thread 0)
  auto issue = [&](int buf) {
    const uint32_t d = tmem + (uint32_t)(buf * Db);
    for (int ks = 0; ks < L / 8; ++ks) {
      const uint64_t a_hi = smem_desc(ah + 256u * ks, 128u, sbo), a_lo = smem_desc(al + 256u * ks, 128u, sbo);
      const uint64_t b_hi = smem_desc(bh + 256u * ks, 128u, sbo), b_lo = smem_desc(bl + 256u * ks, 128u, sbo);
      mma_tf32(d, a_hi, b_hi, idesc, ks > 0 ? 1u : 0u);
      mma_tf32(d, a_lo, b_hi, idesc, 1u);
      mma_tf32(d, a_hi, b_lo, idesc, 1u);
    }
    mma_commit(bar);
  };

  // relevance of a finished tile (first CTA, threads t < 128 = rows) from its norm parts and
  // the prompt dots, or with a partner, its half norm and the dots the partner formed
  auto finish_rel = [&](int64_t tl, int itl) {
    const int64_t pr = tl * kRows + t;
    if (pr >= a.P) return;
    const int nb = itl % kXBufs, db = itl % kDotBufs;
    const float* pb = sPeer + nb * (1 + kMaxText) * kRows + t;   // the partner's row t
    float nrm = 0.f;
    for (int g = 0; g < kGroups; ++g) nrm += sNrm[(nb * kGroups + g) * kRows + t];
    if (nrank > 1) nrm += pb[0];
    const float inv = 1.f / (sqrtf(nrm) + a.eps);
    float d[kMaxText];
#pragma unroll
    for (int j = 0; j < kMaxText; ++j)
      d[j] = j >= ntx ? 0.f : (nrank > 1 ? pb[(1 + j) * kRows] : sDot[(db * kMaxText + j) * kRows + t]);
    float best = 0.f;
#pragma unroll
    for (int j = 1; j < kMaxText; ++j)
      if (j < ntx) best = fmaxf(best, 1.f / (1.f + __expf(a.tau * (d[j] - d[0]) * inv)));
    a.rel[pr] = best;
  };

  // each cluster decodes one contiguous range of tiles (both CTAs the same range)
  const int64_t n_cl = gridDim.x / nrank, cl = blockIdx.x / nrank;
  const int64_t t_per = (n_tiles + n_cl - 1) / n_cl;
  const int64_t t_begin = min(n_tiles, cl * t_per), t_end = min(n_tiles, t_begin + t_per);
  const int n_local = (int)(t_end - t_begin);
  if (n_local > 0) {
    load_rows(t_begin);
    stage_a();
    stage_dots(0);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (n_local > 0 && t == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    issue(0);
  }
  if (n_local > 1) load_rows(t_begin + 1);

  // The exchange of a column-split pair, in kXBufs buffers (tile i in buffer i mod kXBufs):
  // the second CTA stores its 128 half norms into the first CTA's buffer with asynchronous
  // stores that complete the buffer's `full` mbarrier; the first CTA, once it has read them,
  // arrives on the second CTA's `consumed` mbarrier, which the second CTA waits for before
  // it reuses the buffer.  Every wait is bounded (a timeout sets the error flag and ends
  // this thread's part in the exchange).
  // A phase of `full` takes exactly one arrival: thread 0 arms it only while its own waits
  // succeed (a phase it saw complete), never twice.
  auto recv_wait = [&](int i) {   // first CTA: the half norms of tile i are in
    const uint32_t fb = full0 + 8u * (uint32_t)(i % kXBufs);
    if (t == 0 && xfer_ok) mbar_arrive_expect(fb, (uint32_t)((1 + ntx) * kRows * 4));
    if (t < kRows && xfer_ok && !mbar_wait_cluster(fb, (uint32_t)(i / kXBufs) & 1u)) {
      xfer_ok = false;
      if (a.err) atomicExch(a.err, 1);
    }
  };
  auto recv_done = [&](int i) {   // first CTA, after a barrier behind the reads of tile i
    if (t == 0 && i + kXBufs < n_local) mbar_arrive_remote(cluster_addr(cons0 + 8u * (uint32_t)(i % kXBufs), 1u));
  };
  // second CTA, threads t < 128: row t of tile i, its half norm v and (zero = false) the
  // prompt dots it formed for the tile
  auto send = [&](int i, float v, bool zero) {
    if (xfer_ok && i >= kXBufs &&
        !mbar_wait_cluster(cons0 + 8u * (uint32_t)(i % kXBufs), (uint32_t)(i / kXBufs - 1) & 1u)) {
      xfer_ok = false;
      if (a.err) atomicExch(a.err, 1);
    }
    if (xfer_ok) {
      const uint32_t rb = cluster_addr(full0 + 8u * (uint32_t)(i % kXBufs), 0u);
      const float* pb = sPeer + (i % kXBufs) * (1 + kMaxText) * kRows + t;   // the same row there
      st_async_f32(cluster_addr(smem_u32(pb), 0u), v, rb);
      for (int j = 0; j < ntx; ++j)
        st_async_f32(cluster_addr(smem_u32(pb + (1 + j) * kRows), 0u),
                     zero ? 0.f : sDot[((i % kDotBufs) * kMaxText + j) * kRows + t], rb);
    }
  };

  uint32_t phase = 0;
  bool failed = false;
  int done = 0;   // tiles whose epilogue is complete
  for (int it = 0; it < n_local; ++it) {
    const int64_t tile = t_begin + it;
    // the MMAs of this tile are done: A is free and accumulator it & 1 is final
    // (a thread that saw them complete may overwrite their A operand at once; a timeout is
    // made uniform at the staging barrier)
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && it + 1 < n_local) stage_a();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (__syncthreads_or(!ok)) {   // next A staged; every thread takes the same branch
      failed = true;
      break;
    }
    if (it + 1 < n_local && t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue((it + 1) & 1);   // runs during this tile's epilogue
    }
    if (it + 1 < n_local) stage_dots((it + 1) % kDotBufs);
    if (it + 2 < n_local) load_rows(tile + 2);   // consumed after the next tile's MMAs
    if (want_rel && it >= lag) {
      if (exch && rank == 0) recv_wait(it - lag);   // the partner's half norms and dots
      if (rel_here && t < kRows) finish_rel(tile - lag, it - lag);
    }
    // epilogue: TMEM lanes 32 (warp mod 4) .. + 31 = pixels; chunks w / 4, w / 4 + 4, ...
    const int q4 = warp & 3, cg = warp >> 2;
    const int64_t p = tile * kRows + 32 * q4 + lane;
    const bool store = p < a.P && a.F != nullptr;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)((it & 1) * Db);
    float n4[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = 32 * cg; c0 < Dh; c0 += 32 * kGroups) {
      float v[32];
      tmem_ld32(lane_addr + (uint32_t)c0, v);
      const int nv = min(32, Dh - c0);   // a multiple of 16
      if (store) {
        float* fp = a.F + (int64_t)(n_lo + c0) * a.P + p;
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
      sNrm[((it % kXBufs) * kGroups + cg) * kRows + 32 * q4 + lane] = (n4[0] + n4[1]) + (n4[2] + n4[3]);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // accumulator it & 1 read, norms of this tile complete
    if (exch) {
      if (rank == 0 && it >= lag) recv_done(it - lag);
      if (rank == 1 && t < kRows) {
        float s = 0.f;
        for (int g = 0; g < kGroups; ++g) s += sNrm[((it % kXBufs) * kGroups + g) * kRows + t];
        send(it, s, false);
      }
    }
    done = it + 1;
  }
  if (failed) {
    if (t == 0 && a.err) atomicExch(a.err, 1);
    mbar_wait(bar, phase ^ 1u);   // bounded: let this CTA's own MMAs drain before freeing TMEM
  }
  if (exch) {
    // finish the exchange for every tile the partner still sends (zeros after a failure),
    // then meet once more: neither CTA leaves while the other may still address it
    if (rank == 0) {
      for (int i = max(0, done - lag); i < n_local; ++i) {
        recv_wait(i);
        if (!failed && t < kRows) finish_rel(t_begin + i, i);
        __syncthreads();
        recv_done(i);
      }
    } else if (t < kRows) {
      for (int i = done; i < n_local; ++i) send(i, 0.f, true);
    }
    __syncwarp();
    cluster_arrive();
    cluster_wait();
  } else if (!failed && rel_here && t < kRows && n_local > 0) {
    finish_rel(t_end - 1, n_local - 1);
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

size_t decode_smem(int L, int Dh) { return DecodeSmem(L, Dh).total; }

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
  // Up to 256 columns one CTA holds the split codebook; above, a cluster of two splits the
  // columns (the first takes the larger share, a multiple of 16 for the MMA's N).
  const int nc = Dc <= kMaxDh ? 1 : 2;
  const int Dh0 = nc == 1 ? Dc : std::min(kMaxDh, (Dc / 2 + 15) / 16 * 16);
  // Each CTA holds two accumulators of Db columns.  At most 512 / ncols CTAs may hold their
  // tensor memory on one SM at a time: request enough shared memory that no more than that
  // many are resident (a further CTA would only wait inside its allocation).
  const int Db = (Dh0 + 31) / 32 * 32;
  int ncols = 32;
  while (ncols < 2 * Db) ncols <<= 1;
  const int per_sm = 512 / ncols;
  size_t smem = decode_smem(L, Dh0);
  if (per_sm < kMaxResident && smem_sm > 0)
    smem = std::max<size_t>(smem, (size_t)smem_sm / (size_t)(per_sm + 1) + 1024);
  if (cudaFuncSetAttribute(k_vq_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return GS_ERR_CUDA;
  DecodeArgs a{wmap, P, L, codebook, Dc, Dh0, F_out, text, relevance ? n_text : 0, tau, 1e-8f,
               relevance, err};
  const int64_t n_tiles = (P + kRows - 1) / kRows;
  const int64_t clusters = min64(n_tiles, (int64_t)sms * per_sm / nc);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(clusters * nc), 1, 1);
  cfg.blockDim = dim3(kVT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_vq_decode, a);
  note_launch();
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
