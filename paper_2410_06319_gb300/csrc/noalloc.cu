// lsq_qr_r_noalloc: the Householder QR of a sketch (Algorithm 1 (the QR of the sketch)) run
// entirely in a fixed, file-scope device scratch array, for callers that must
// not allocate (see include/lsq.h).  The factorization itself is the same
// launch sequence lsq_qr_r uses; only where its scratch lives differs.
//
// Scratch layout (one copy per device, 256-byte aligned):
//   [0, kWorkBytes)                 working copy of Y (s x (n+1), FP32 or FP64)
//   [kWorkBytes, +kAuxBytes)        norms, diag(R), tau and the compact-WY T factor
//   [kWorkBytes + kAuxBytes, +256)  grid-barrier counter and generation word
//                                   (two unsigned), then the error word (int)
// Must start at zero on every call: the two barrier words and the error word.
// The call clears them on the caller's stream before its first kernel; every
// other byte is written before it is read.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "lsq.h"

namespace {

constexpr size_t kWorkBytes = (size_t)LSQ_NOALLOC_WORK_BYTES;
constexpr size_t kAuxBytes = 64 * 1024;
constexpr size_t kWordBytes = 256;
constexpr size_t kScratchBytes = kWorkBytes + kAuxBytes + kWordBytes;
constexpr int kMaxDevices = 64;
constexpr int kErrRank = 100;   // a zero or non-finite diagonal entry of R

__device__ __align__(256) unsigned char g_qr_scratch[kScratchBytes];

struct DeviceScratch {
  unsigned char* base = nullptr;
  int num_sms = 0;
};

std::mutex g_setup_mu;
DeviceScratch g_dev[kMaxDevices];

// Once per device, with that device current: the address of this device's copy
// of the scratch array and its SM count.
lsq_status scratch_for_current_device(DeviceScratch* out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSQ_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LSQ_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceScratch& d = g_dev[dev];
  if (!d.base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qr_scratch) != cudaSuccess || !p) return LSQ_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return LSQ_E_CUDA;
    d.num_sms = sms;
    d.base = static_cast<unsigned char*>(p);
  }
  *out = d;
  return LSQ_OK;
}

// R (normalised to diag >= 0 by the finalize step) must have a positive,
// finite diagonal.
__global__ void diag_check_kernel(const double* __restrict__ R, int64_t n, int* err) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = R[i * n + i];
    if (!(d > 0.0) || !isfinite(d)) lsq::set_error(err, kErrRank);
  }
}

}  // namespace

extern "C" lsq_status lsq_qr_r_noalloc(const double* Y, int64_t s, int64_t n, lsq_prec u_p, double* R,
                                       double* c, void* cuda_stream) {
  if (!Y || !R || n < 1 || s < n || s > 16384) return LSQ_E_INVAL;
  if (u_p != LSQ_F32 && u_p != LSQ_F64) return LSQ_E_INVAL;
  const bool f64 = (u_p == LSQ_F64);
  const int64_t elem = f64 ? 8 : 4;
  if (n > LSQ_NOALLOC_MAX_N || s > (int64_t)(kWorkBytes / (size_t)elem) / (n + 1)) return LSQ_E_SIZE;
  DeviceScratch d;
  const lsq_status sv = scratch_for_current_device(&d);
  if (sv != LSQ_OK) return sv;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* work = d.base;
  double* aux = reinterpret_cast<double*>(d.base + kWorkBytes);
  unsigned* bar = reinterpret_cast<unsigned*>(d.base + kWorkBytes + kAuxBytes);
  int* err = reinterpret_cast<int*>(bar + 2);
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned) + sizeof(int), st) != cudaSuccess) return LSQ_E_CUDA;
  if (lsq::launch_qr(f64, Y, s, n, work, aux, bar, R, c, err, d.num_sms, st) != cudaSuccess)
    return LSQ_E_CUDA;
  diag_check_kernel<<<1, 256, 0, st>>>(R, n, err);
  if (cudaGetLastError() != cudaSuccess) return LSQ_E_CUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LSQ_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LSQ_E_CUDA;
  if (herr == lsq::DEV_TIMEOUT_GRID) return LSQ_E_TIMEOUT;
  if (herr == kErrRank) return LSQ_E_RANK;
  if (herr != 0) return LSQ_E_CUDA;
  return LSQ_OK;
}
