// FMA issue-rate microbenchmark: the FP32 and FP64 pipe peaks of the device,
// measured with independent dependent-FMA chains per thread, so that the
// pair passes (bound by plain FP arithmetic, not by a dense contraction) can
// be stated as a fraction of a measured pipe peak.
#include "sph_kernels.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ double g_sink;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-1.2345) g_sink = (double)s;  // never true; keeps the chains alive
}

template <class T>
sph_status run(int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPH_ERR_CUDA;
  const int blocks = sms * 8;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return SPH_ERR_CUDA;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SPH_ERR_CUDA;
  const T b = (T)0.999999, c = (T)1e-6;
  k_fma_chain<T><<<blocks, kThreads, 0, s>>>(iters / 8, b, c);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_chain<T><<<blocks, kThreads, 0, s>>>(iters, b, c);
  cudaEventRecord(e1, s);
  sph_status st = SPH_OK;
  float ms = 0.f;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    st = SPH_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) st = SPH_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st != SPH_OK) return st;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_fma_peak(int32_t precision, int32_t iters, double* tflops) {
  if (!tflops || iters < 64) return SPH_ERR_ARG;
  if (precision == SPH_FP64) return run<double>(iters, tflops);
  if (precision == SPH_MIXED) return run<float>(iters, tflops);
  return SPH_ERR_ARG;
}
