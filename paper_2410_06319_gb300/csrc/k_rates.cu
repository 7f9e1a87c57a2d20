// Throughput probes for the rooflines of ALU-bound kernels: the FP64 (and FP32)
// fused multiply-add rate of the device, measured with independent FMA chains in
// every thread of a grid that fills every SM.
#include <cuda_runtime.h>

#include "lsq.h"

namespace {

constexpr int kChains = 8;       // independent accumulators per thread (hides the FMA latency)
constexpr int kIters = 4096;     // FMAs per chain
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T x, T y, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], x, y);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)1234.5) out[0] = s;   // keeps the chains live; never true for the inputs used
}

template <typename T>
lsq_status measure(cudaStream_t st, double* fma_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LSQ_E_CUDA;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return LSQ_E_NOMEM;
  lsq_status rc = LSQ_OK;
  const unsigned blocks = (unsigned)sms * 8u;
  double best = 0.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = LSQ_E_CUDA;
  for (int rep = 0; rep < 6 && rc == LSQ_OK; ++rep) {
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<blocks, kThreads, 0, st>>>((T)0.999999, (T)1e-7, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = LSQ_E_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double r = (double)blocks * kThreads * kIters * kChains / (ms * 1e-3);
    if (rep > 0 && r > best) best = r;   // the first launch is a warm-up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == LSQ_OK) *fma_per_s = best;
  return rc;
}

}  // namespace

extern "C" lsq_status lsq_probe_fma_rate(int which, void* cuda_stream, double* fma_per_s) {
  if (!fma_per_s) return LSQ_E_INVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (which == 0) return measure<double>(st, fma_per_s);
  if (which == 1) return measure<float>(st, fma_per_s);
  return LSQ_E_INVAL;
}
