// FP32 FMA throughput of the current GPU, measured.
//
// The rasterizer kernels (a3/a4) are bound by plain FP32 arithmetic, not by HBM or the
// tensor cores, so their roofline needs the FP32 peak of the part as it runs: this kernel
// fills every SM to its occupancy limit with threads that each advance eight independent
// x <- x * a + b chains (fmaf, one instruction = 2 FLOPs) and is timed with CUDA events on
// the caller's stream.  It only reads a few scalars and writes nothing unless a value
// that cannot occur appears, and it changes no setting of the GPU.
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

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_measure_fp32_peak(int iters, double* tflops_out, double* ms_out,
                                          void* stream) {
  if (iters <= 0 || !tflops_out) return GS_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0) !=
          cudaSuccess)
    return GS_ERR_CUDA;
  if (per_sm < 1) return GS_ERR_CUDA;
  const int blocks = sms * per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GS_ERR_CUDA;
  }
  const float a = 0.999999f, b = 1e-6f;
  // one short launch to warm up, then the timed one
  k_fma_peak<<<blocks, kPeakThreads, 0, st>>>(nullptr, a, b, iters / 16 + 1);
  cudaEventRecord(e0, st);
  k_fma_peak<<<blocks, kPeakThreads, 0, st>>>(nullptr, a, b, iters);
  cudaEventRecord(e1, st);
  note_launch(2);
  float ms = 0.f;
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return GS_ERR_CUDA;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kPeakThreads;
  *tflops_out = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return GS_OK;
}
