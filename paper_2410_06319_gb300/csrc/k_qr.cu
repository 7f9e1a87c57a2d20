// Algorithm 1 step 2: Householder QR of the sketch Y (s x n) in precision
// u_QR (FP32 or FP64), R factor only; the reflectors are also applied to the
// sketched right-hand side (column n), giving c = (Q^T Omega b)[:n] for the
// sketch-and-solve start x_s = R^-1 c (Sec. 4).
//
// Reflector k (Golub & Van Loan): x = W[k:, k], alpha = ||x||, v = x + sign(x_1)
// alpha e_1, H = I - v v^T / (alpha (alpha + |x_1|)); R_kk = -sign(x_1) alpha.
// One cooperative launch runs all n steps; per step every block loads v into
// shared memory, each block updates whole trailing columns (block-wide
// reductions), the block owning column k+1 also leaves its squared norm for
// the next step, and a bounded grid barrier separates the steps.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace lsq {

template <typename T>
__device__ __forceinline__ T block_sum_256(T v, T* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  return red[32];
}

template <typename T>
__global__ void convert_y_kernel(const double* __restrict__ Y, T* __restrict__ W, int64_t total) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < total) W[i] = (T)Y[i];
}

template <typename T>
__global__ void __launch_bounds__(256) qr_kernel(T* __restrict__ W, int64_t s, int64_t n,
                                                 double* __restrict__ norms,
                                                 double* __restrict__ diagR, unsigned* bar,
                                                 int* err) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  T* vs = reinterpret_cast<T*>(qr_smem);
  __shared__ T red[33];
  const unsigned nb = gridDim.x;
  if (blockIdx.x == 0) {
    T part = 0;
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) part += W[t] * W[t];
    const T nn = block_sum_256(part, red);
    if (threadIdx.x == 0) norms[0] = (double)nn;
  }
  if (!grid_barrier(bar, bar + 1, nb, err)) return;
  for (int64_t k = 0; k < n; ++k) {
    const T* colk = W + k * s;
    const T alpha = sqrt((T)norms[k]);
    const T x0 = colk[k];
    const T sgn = (x0 >= T(0)) ? T(1) : T(-1);
    const T scale = (alpha > T(0)) ? T(1) / (alpha * (alpha + fabs(x0))) : T(0);
    if (blockIdx.x == 0 && threadIdx.x == 0) diagR[k] = (double)(-sgn * alpha);
    const int64_t len = s - k;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) vs[t] = (t == 0) ? x0 + sgn * alpha : colk[k + t];
    __syncthreads();
    for (int64_t j = k + 1 + blockIdx.x; j <= n; j += nb) {
      T* colj = W + j * s + k;
      T part = 0;
      for (int64_t t = threadIdx.x; t < len; t += blockDim.x) part += vs[t] * colj[t];
      const T wj = block_sum_256(part, red) * scale;
      T part2 = 0;
      for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
        const T val = colj[t] - wj * vs[t];
        colj[t] = val;
        if (t >= 1) part2 += val * val;
      }
      if (j == k + 1 && j < n) {
        const T nn = block_sum_256(part2, red);
        if (threadIdx.x == 0) norms[k + 1] = (double)nn;
      }
    }
    if (!grid_barrier(bar, bar + 1, nb, err)) return;
  }
}

// R (FP64, col-major, diag >= 0) and c from the factored work matrix.
template <typename T>
__global__ void qr_finalize_kernel(const T* __restrict__ W, int64_t s, int64_t n,
                                   const double* __restrict__ diagR, double* __restrict__ R,
                                   double* __restrict__ c) {
  const int64_t j = blockIdx.x;          // column of R
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double sg = (diagR[i] < 0.0) ? -1.0 : 1.0;
    double v = 0.0;
    if (i == j) v = diagR[i];
    else if (i < j) v = (double)W[j * s + i];
    if (R) R[j * n + i] = v * sg;
    if (c && j == 0) c[i] = (double)W[n * s + i] * sg;
  }
}

template <typename T>
static cudaError_t run_qr(const double* Y, int64_t s, int64_t n, T* W, double* aux, unsigned* bar,
                          double* R, double* c, int* err, int num_sms, cudaStream_t st) {
  const int64_t total = s * (n + 1);
  convert_y_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Y, W, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)s * sizeof(T);
  auto kern = qr_kernel<T>;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)occ * num_sms;
  if (grid > n) grid = n;
  if (grid < 1) grid = 1;
  double* norms = aux;
  double* diagR = aux + n;
  T* Wp = W;
  int64_t sp = s, np = n;
  void* args[] = {&Wp, &sp, &np, &norms, &diagR, &bar, &err};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(256), args, smem, st);
  if (e != cudaSuccess) return e;
  qr_finalize_kernel<T><<<(unsigned)n, 256, 0, st>>>(W, s, n, diagR, R, c);
  return cudaGetLastError();
}

cudaError_t launch_qr(bool fp64, const double* Y, int64_t s, int64_t n, void* work, double* aux,
                      unsigned* bar, double* R, double* c, int* err, int num_sms, cudaStream_t st) {
  if (fp64)
    return run_qr<double>(Y, s, n, static_cast<double*>(work), aux, bar, R, c, err, num_sms, st);
  return run_qr<float>(Y, s, n, static_cast<float*>(work), aux, bar, R, c, err, num_sms, st);
}

}  // namespace lsq
