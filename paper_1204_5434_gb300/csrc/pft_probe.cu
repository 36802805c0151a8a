// pft_probe.cu -- fused multiply-add throughput of the GPU the library runs on.
//
// The FP64 path of the contour step is bound by the FP64 pipe, not by HBM, so its
// roofline denominator is the DFMA rate of the device it runs on; the FP32 rate is
// measured the same way for comparison.  One launch of independent FMA chains over
// every SM, timed with CUDA events after a warm-up launch.
#include <string>

#include "pft_engine.h"

namespace pft {
namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_loop(T* __restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += x[j];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;  // keeps every chain live
}

template <typename T>
cudaError_t fma_rate(int iters, double* tflops, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * kBlocksPerSm;
  T* out = nullptr;
  e = cudaMallocAsync((void**)&out, (size_t)blocks * kThreads * sizeof(T), stream);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a contraction towards the fixed point b / (1 - a): the chains stay finite
  const T a = (T)0.999, b = (T)1e-3;
  if (e == cudaSuccess) {
    k_fma_loop<T><<<blocks, kThreads, 0, stream>>>(out, iters, a, b);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
  if (e == cudaSuccess) {
    k_fma_loop<T><<<blocks, kThreads, 0, stream>>>(out, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) {
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t e2 = cudaFreeAsync(out, stream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

}  // namespace
}  // namespace pft

extern "C" pft_status pft_fma_throughput(int precision, double* tflops, void* stream) {
  if (!tflops) {
    pft::set_error("pft_fma_throughput: tflops is NULL");
    return PFT_ERR_ARG;
  }
  if (precision != PFT_FP64 && precision != PFT_FP32_MIXED) {
    pft::set_error("pft_fma_throughput: unknown precision");
    return PFT_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // about 20 ms per launch on GB300 at either rate (FP32 runs 64x the FP64 rate)
  cudaError_t e = (precision == PFT_FP64) ? pft::fma_rate<double>(4096, tflops, s)
                                          : pft::fma_rate<float>(4096 * 64, tflops, s);
  if (e != cudaSuccess) {
    pft::set_error(std::string("pft_fma_throughput: ") + cudaGetErrorString(e));
    return PFT_ERR_CUDA;
  }
  return PFT_OK;
}
