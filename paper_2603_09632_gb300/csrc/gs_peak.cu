// FP32 FMA throughput of the current GPU, measured.
//
// The rasterizer kernels (a3/a4) are bound by plain FP32 arithmetic, not by HBM or the
// tensor cores, so their roofline needs the FP32 peak of the part as it runs: these kernels
// fill every SM to its occupancy limit with threads that each advance eight independent
// x <- x * a + b chains, once as scalar fmaf and once as packed pairs (fma.rn.f32x2, two
// FMAs per instruction, which the raster kernels use for their accumulations), and are
// timed with CUDA events on the caller's stream; the larger rate is the peak.  They only
// read a few scalars and write nothing unless a value that cannot occur appears, and they
// change no setting of the GPU.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kPeakThreads = 512;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* sink, float a, float b, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a, b keep every chain near b / (1 - a) = 1; the store never happens but the compiler
  // cannot prove it, so the chains are not removed
  if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same kChains chains per thread as kChains / 2 packed pairs.
__global__ void __launch_bounds__(kPeakThreads) k_fma2_peak(float* sink, float a, float b, int iters) {
  float2 x[kChains / 2];
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c)
    x[c] = make_float2((float)(threadIdx.x + 2 * c) * 1e-6f, (float)(threadIdx.x + 2 * c + 1) * 1e-6f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
  if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warm-up launch, then one timed launch (ms), of a peak kernel on every SM.
template <typename K>
bool time_peak(K kern, int sms, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int* blocks,
               float* ms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeakThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return false;
  *blocks = sms * per_sm;
  const float a = 0.999999f, b = 1e-6f;
  kern<<<*blocks, kPeakThreads, 0, st>>>(nullptr, a, b, iters / 16 + 1);
  cudaEventRecord(e0, st);
  kern<<<*blocks, kPeakThreads, 0, st>>>(nullptr, a, b, iters);
  cudaEventRecord(e1, st);
  note_launch(2);
  *ms = 0.f;
  return cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(ms, e0, e1) == cudaSuccess && *ms > 0.f;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_measure_fp32_peak(int iters, double* tflops_out, double* ms_out,
                                          void* stream) {
  if (iters <= 0 || !tflops_out) return GS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GS_ERR_CUDA;
  }
  int blocks1 = 0, blocks2 = 0;
  float ms1 = 0.f, ms2 = 0.f;
  const bool ok = time_peak(k_fma_peak, sms, iters, st, e0, e1, &blocks1, &ms1) &&
                  time_peak(k_fma2_peak, sms, iters, st, e0, e1, &blocks2, &ms2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return GS_ERR_CUDA;
  const double per_thread = 2.0 * kChains * kUnroll * (double)iters * kPeakThreads;
  const double t1 = per_thread * blocks1 / (ms1 * 1e-3) / 1e12, t2 = per_thread * blocks2 / (ms2 * 1e-3) / 1e12;
  *tflops_out = t1 > t2 ? t1 : t2;
  if (ms_out) *ms_out = t1 > t2 ? ms1 : ms2;
  return GS_OK;
}
