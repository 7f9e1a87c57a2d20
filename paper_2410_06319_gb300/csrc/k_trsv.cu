// Triangular solves with the sketched R (Alg. 2: x_s = R^-1 c, the right
// preconditioner R^-1 in LSQR and FGMRES, the left preconditioner R^-T, and
// h = R^-T g in u_r).
//
// One CTA of 1024 threads, the right-hand side in shared memory, blocks of 32
// rows.  The inverses of the 32 x 32 diagonal blocks are formed once per R
// (dinv_kernel), so a block step is a 32 x 32 matrix-vector product by warp 0
// followed by a rank-32 update of the remaining rows by all threads; there is
// no serial substitution chain inside a block.  The matrices are R (upper) and
// L = R^T (lower), both column-major, so every update reads contiguous column
// segments, which cp.async stages into shared memory ahead of the step that
// uses them (trsv.cuh).
#include "common.cuh"
#include "kernels.h"
#include "trsv.cuh"

namespace lsq {

template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_kernel(const T* __restrict__ M, int64_t ld, const T* __restrict__ D, int n,
                const TIN* __restrict__ y, double yscale, TOUT* __restrict__ x, const int* done,
                const int* jp, int64_t ys, int64_t xstr, int* err) {
  if (done && *done) return;
  if (jp) {  // column j of a basis: offsets read on the device (graph-replayable)
    const int64_t j = *jp;
    y += j * ys;
    x += j * xstr;
  }
  __shared__ T xs[1024];
  extern __shared__ __align__(16) unsigned char trsv_buf[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (T)((double)y[i] * yscale);
  __syncthreads();
  if (!block_trsv<T, UPPER>(M, ld, D, n, xs, trsv_buf, err)) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = (TOUT)xs[i];
}

template <typename T, typename TIN, typename TOUT>
cudaError_t launch_trsv(bool upper, const Tri<T>& f, const TIN* y, double yscale, TOUT* x,
                        const int* done, cudaStream_t st, const int* jp, int64_t ys, int64_t xstr) {
  if (f.n > 1024) return cudaErrorInvalidValue;
  const size_t smem = TrsvSmem<T>::bytes;
  if (upper) {
    auto kern = trsv_kernel<T, TIN, TOUT, true>;
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kTrsvThreads, smem, st>>>(f.R, f.ld, f.DU, (int)f.n, y, yscale, x, done, jp, ys, xstr, f.err);
  } else {
    auto kern = trsv_kernel<T, TIN, TOUT, false>;
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kTrsvThreads, smem, st>>>(f.L, f.ld, f.DL, (int)f.n, y, yscale, x, done, jp, ys, xstr, f.err);
  }
  return cudaGetLastError();
}

#define LSQ_TRSV_INST(T, TIN, TOUT)                                                                  \
  template cudaError_t launch_trsv<T, TIN, TOUT>(bool, const Tri<T>&, const TIN*, double, TOUT*,  \
                                                 const int*, cudaStream_t, const int*, int64_t,   \
                                                 int64_t);
LSQ_TRSV_INST(float, float, float)
LSQ_TRSV_INST(float, double, float)
LSQ_TRSV_INST(float, float, double)
LSQ_TRSV_INST(float, double, double)
LSQ_TRSV_INST(double, double, double)
LSQ_TRSV_INST(double, float, double)
LSQ_TRSV_INST(double, double, float)
LSQ_TRSV_INST(double, float, float)

// ------------------------------------------------------------ preparation
__global__ void prepare_r_kernel(const double* __restrict__ R, int64_t n, float* R32, float* L32,
                                 int64_t ld32, double* R64, double* L64, int64_t ld64) {
  const int64_t j = blockIdx.x;
  for (int64_t i = threadIdx.x; i < ld32; i += blockDim.x) {
    const double v = (i <= j && i < n) ? R[j * n + i] : 0.0;   // R(i, j), upper
    R32[j * ld32 + i] = (float)v;
    if (i < n) L32[i * ld32 + j] = (float)v;                  // L(j, i) = R(i, j)
    else L32[j * ld32 + i] = 0.0f;                            // padding rows of L's column j
  }
  for (int64_t i = threadIdx.x; i < ld64; i += blockDim.x) {
    const double v = (i <= j && i < n) ? R[j * n + i] : 0.0;
    R64[j * ld64 + i] = v;
    if (i < n) L64[i * ld64 + j] = v;
    else L64[j * ld64 + i] = 0.0;
  }
}

// Inverse of the diagonal block k of the upper-triangular R (one warp per
// block): lane j forms column j of T^-1 by back substitution.  DU(i, j) at
// k*1024 + j*32 + i; DL = DU^T (the inverse of the diagonal block of R^T) at
// k*1024 + i*32 + j.
template <typename T>
__global__ void dinv_kernel(const T* __restrict__ R, int64_t ld, int n, T* __restrict__ DU,
                            T* __restrict__ DL) {
  __shared__ T tb[32][33];
  const int k = blockIdx.x, lane = threadIdx.x;
  const int i0 = k * 32, w = min(32, n - i0);
  for (int c = 0; c < 32; ++c) tb[lane][c] = (lane < w && c < w) ? R[(size_t)(i0 + c) * ld + i0 + lane] : T(0);
  __syncwarp();
  T x[32];
#pragma unroll
  for (int i = 31; i >= 0; --i) {
    T t = (i == lane) ? T(1) : T(0);
#pragma unroll
    for (int c = i + 1; c < 32; ++c) t -= tb[i][c] * x[c];
    x[i] = (i < w && lane < w) ? t / tb[i][i] : T(0);
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    DU[(size_t)k * 1024 + lane * 32 + i] = x[i];
    DL[(size_t)k * 1024 + i * 32 + lane] = x[i];
  }
}

__global__ void kappa_diag_kernel(const double* __restrict__ R, int64_t n, double* out) {
  __shared__ double mx[32], mn[32];
  double a = 0.0, b = INFINITY;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = fabs(R[i * n + i]);
    if (!(d < INFINITY)) bad = true;
    a = fmax(a, d);
    b = fmin(b, d);
  }
  if (bad) b = 0.0;
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

cudaError_t launch_prepare_r(const double* R, int64_t n, Tri<float>* f32, Tri<double>* f64,
                             double* kappa_est, cudaStream_t st) {
  prepare_r_kernel<<<(unsigned)n, 256, 0, st>>>(R, n, const_cast<float*>(f32->R), const_cast<float*>(f32->L),
                                                f32->ld, const_cast<double*>(f64->R),
                                                const_cast<double*>(f64->L), f64->ld);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((n + 31) / 32);
  dinv_kernel<float><<<nb, 32, 0, st>>>(f32->R, f32->ld, (int)n, const_cast<float*>(f32->DU),
                                        const_cast<float*>(f32->DL));
  dinv_kernel<double><<<nb, 32, 0, st>>>(f64->R, f64->ld, (int)n, const_cast<double*>(f64->DU),
                                         const_cast<double*>(f64->DL));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (kappa_est) {
    kappa_diag_kernel<<<1, 256, 0, st>>>(R, n, kappa_est);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace lsq
