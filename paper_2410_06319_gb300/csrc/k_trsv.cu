// Triangular solves with the sketched R (Alg. 2: x_s = R^-1 c, the right
// preconditioner R^-1 in LSQR and FGMRES, the left preconditioner R^-T, and
// h = R^-T g in u_r).
//
// One CTA of 1024 threads; the right-hand side lives in shared memory.  The
// matrix is upper R or L = R^T, both column-major, so every access below reads
// contiguous column segments.  Blocks of 32 rows: warp 0 holds the 32 x 32
// diagonal block in registers (one row per lane) and substitutes serially,
// then all threads subtract the block's contribution from the remaining rows.
#include "common.cuh"
#include "kernels.h"

namespace lsq {

constexpr int kTrsvThreads = 1024;

template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_kernel(const T* __restrict__ M, int n, const TIN* __restrict__ y, double yscale,
                TOUT* __restrict__ x, const int* done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char trsv_smem[];
  T* xs = reinterpret_cast<T*>(trsv_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) xs[i] = (T)((double)y[i] * yscale);
  __syncthreads();
  const int nb = (n + 31) >> 5;
  for (int bi = 0; bi < nb; ++bi) {
    const int ib = UPPER ? nb - 1 - bi : bi;
    const int i0 = ib * 32;
    const int w = min(32, n - i0);
    if (warp == 0) {
      T d[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        d[jj] = (jj < w && lane < w) ? M[(int64_t)(i0 + jj) * n + i0 + lane] : T(0);
      T xl = (lane < w) ? xs[i0 + lane] : T(0);
      if (UPPER) {
#pragma unroll
        for (int jj = 31; jj >= 0; --jj) {
          if (jj < w) {
            if (lane == jj) xl = xl / d[jj];
            const T xj = __shfl_sync(0xffffffffu, xl, jj);
            if (lane < jj) xl -= d[jj] * xj;
          }
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          if (jj < w) {
            if (lane == jj) xl = xl / d[jj];
            const T xj = __shfl_sync(0xffffffffu, xl, jj);
            if (lane > jj) xl -= d[jj] * xj;
          }
        }
      }
      if (lane < w) xs[i0 + lane] = xl;
    }
    __syncthreads();
    if (UPPER) {
      for (int r = tid; r < i0; r += blockDim.x) {
        T acc = 0;
        for (int c = i0; c < i0 + w; ++c) acc += M[(int64_t)c * n + r] * xs[c];
        xs[r] -= acc;
      }
    } else {
      for (int r = i0 + w + tid; r < n; r += blockDim.x) {
        T acc = 0;
        for (int c = i0; c < i0 + w; ++c) acc += M[(int64_t)c * n + r] * xs[c];
        xs[r] -= acc;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) x[i] = (TOUT)xs[i];
}

template <typename T, typename TIN, typename TOUT>
cudaError_t launch_trsv(bool upper, const T* M, int64_t n, const TIN* y, double yscale, TOUT* x,
                        const int* done, cudaStream_t st) {
  const size_t smem = (size_t)n * sizeof(T);
  if (upper)
    trsv_kernel<T, TIN, TOUT, true><<<1, kTrsvThreads, smem, st>>>(M, (int)n, y, yscale, x, done);
  else
    trsv_kernel<T, TIN, TOUT, false><<<1, kTrsvThreads, smem, st>>>(M, (int)n, y, yscale, x, done);
  return cudaGetLastError();
}

#define LSQ_TRSV_INST(T, TIN, TOUT)                                                          \
  template cudaError_t launch_trsv<T, TIN, TOUT>(bool, const T*, int64_t, const TIN*, double, \
                                                 TOUT*, const int*, cudaStream_t);
LSQ_TRSV_INST(float, float, float)
LSQ_TRSV_INST(float, double, float)
LSQ_TRSV_INST(float, float, double)
LSQ_TRSV_INST(float, double, double)
LSQ_TRSV_INST(double, double, double)
LSQ_TRSV_INST(double, float, double)
LSQ_TRSV_INST(double, double, float)
LSQ_TRSV_INST(double, float, float)

__global__ void prepare_r_kernel(const double* __restrict__ R, int64_t n, float* R32, float* L32,
                                 double* R64, double* L64) {
  const int64_t j = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = (i <= j) ? R[j * n + i] : 0.0;   // R(i, j), upper
    if (R32) R32[j * n + i] = (float)v;
    if (R64) R64[j * n + i] = v;
    // L = R^T column-major: L(j, i) at i * n + j
    if (L32) L32[i * n + j] = (float)v;
    if (L64) L64[i * n + j] = v;
  }
}

__global__ void kappa_diag_kernel(const double* __restrict__ R, int64_t n, double* out) {
  __shared__ double mx[32], mn[32];
  double a = 0.0, b = INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = fabs(R[i * n + i]);
    a = fmax(a, d);
    b = fmin(b, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmin(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    mx[warp] = a;
    mn[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = fmax(a, mx[w]);
      b = fmin(b, mn[w]);
    }
    *out = (b > 0.0) ? a / b : INFINITY;
  }
}

cudaError_t launch_prepare_r(const double* R, int64_t n, float* R32, float* L32, double* R64,
                             double* L64, double* kappa_est, cudaStream_t st) {
  prepare_r_kernel<<<(unsigned)n, 256, 0, st>>>(R, n, R32, L32, R64, L64);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (kappa_est) {
    kappa_diag_kernel<<<1, 256, 0, st>>>(R, n, kappa_est);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace lsq
