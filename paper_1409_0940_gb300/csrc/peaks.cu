// Measured FMA throughput of the SIMT pipes (FP32 and FP64): the denominators of the rooflines
// of the SIMT kernels (the FP32 regeneration passes, the set-up GEMMs).  Each thread runs eight
// independent multiply-add chains x <- x b + c (|b| < 1, so the values stay bounded), enough
// independent work to cover the pipe latency at four 256-thread CTAs per SM.
#include "common.cuh"
#include "internal.h"
#include "rff_admm.h"

namespace rff {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(const T* __restrict__ in, T* __restrict__ out, int iters) {
  const T b = in[0], c = in[1];
  T x0 = in[2] + (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3, x4 = x0 + (T)4, x5 = x0 + (T)5,
    x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, b, c);
    x1 = fma(x1, b, c);
    x2 = fma(x2, b, c);
    x3 = fma(x3, b, c);
    x4 = fma(x4, b, c);
    x5 = fma(x5, b, c);
    x6 = fma(x6, b, c);
    x7 = fma(x7, b, c);
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == in[3]) out[blockIdx.x] = s;   // never equal: keeps the chains without a store per thread
}

template <typename T>
cudaError_t time_chains(int iters, cudaStream_t st, double* tflops) {
  int sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)sms * 4;
  T* buf = nullptr;
  if ((e = cudaMallocAsync((void**)&buf, (4 + grid) * sizeof(T), st)) != cudaSuccess) return e;
  const T init[4] = {(T)0.999, (T)0.001, (T)0.5, (T)-12345.0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_chains<T><<<grid, 256, 0, st>>>(buf, buf + 4, iters / 8);   // warm-up (clocks, caches)
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<grid, 256, 0, st>>>(buf, buf + 4, iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) *tflops = 2.0 * 8.0 * (double)grid * 256.0 * (double)iters / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  return e;
}

}  // namespace
}  // namespace rff

extern "C" rff_status rff_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* stream) {
  if (!fp32_tflops || !fp64_tflops) return RFF_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (rff::time_chains<float>(1 << 19, st, fp32_tflops) != cudaSuccess) return RFF_ECUDA;
  if (rff::time_chains<double>(1 << 13, st, fp64_tflops) != cudaSuccess) return RFF_ECUDA;
  return RFF_OK;
}
