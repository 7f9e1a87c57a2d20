// Algorithm 1 (the QR of the sketch): Householder QR of the sketch Y (s x n) in precision
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
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"
#include "batch.h"
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

// FP64 variant (u_QR = double) for GB300's narrow FP64 pipe: one 512-thread CTA per SM.
// Step k: every CTA loads v_k into shared memory; CTA b takes a contiguous share of the
// trailing columns k+1..n (column n is Omega b) and treats them eight at a time: one sweep
// over the rows forms the eight dot products v^T y_j (eight independent FMA chains per
// thread), one reduce-scatter butterfly per warp and sixteen-term sums give w_j, and a
// second sweep applies y_j -= (w_j tau) v (the owner of column k+1 also sums the squares of
// its updated rows 1.. for the next norm).  One bounded grid barrier per step, as before;
// the same reflectors and per-column arithmetic, with blocked sums.
constexpr int kQr64Threads = 512;

__global__ void __launch_bounds__(kQr64Threads, 1)
    qr64_kernel(double* __restrict__ W, int64_t s, int64_t n, double* __restrict__ norms,
                double* __restrict__ diagR, unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  double* vs = reinterpret_cast<double*>(qr_smem);
  __shared__ double red[16 * 9];
  __shared__ double wsum[8];
  __shared__ double nred[17];
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (blockIdx.x == 0) {
    double part = 0.0;
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) part = fma(W[t], W[t], part);
    part = warp_sum(part);
    if (lane == 0) nred[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double q = 0.0;
      for (int w = 0; w < nw; ++w) q += nred[w];
      norms[0] = q;
    }
  }
  if (!grid_barrier(bar, bar + 1, nb, err)) return;
  for (int64_t k = 0; k < n; ++k) {
    const double* colk = W + k * s;
    const double alpha = sqrt(__ldcg(norms + k));
    const double x0 = __ldcg(colk + k);
    const double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
    const double tau = (alpha > 0.0) ? 1.0 / (alpha * (alpha + fabs(x0))) : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) diagR[k] = -sgn * alpha;
    const int64_t len = s - k;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) vs[t] = (t == 0) ? x0 + sgn * alpha : __ldcg(colk + k + t);
    __syncthreads();
    const int64_t ntr = n - k;                       // trailing columns k+1..n
    const int64_t per = (ntr + nb - 1) / nb;
    const int64_t j0 = k + 1 + (int64_t)blockIdx.x * per, j1 = min(n + 1, j0 + per);
    for (int64_t g = j0; g < j1; g += 8) {
      double d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = 0.0;
      for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
        const double vt = vs[t];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (g + q < j1) d[q] = fma(vt, __ldcg(W + (g + q) * s + k + t), d[q]);
      }
      const double tot = warp_reduce8(d);
      if ((lane & 3) == 0) red[warp * 9 + ((lane >> 2) & 7)] = tot;
      __syncthreads();
      if (threadIdx.x < 8) {
        double q = 0.0;
        for (int w = 0; w < nw; ++w) q += red[w * 9 + threadIdx.x];
        wsum[threadIdx.x] = q * tau;
      }
      __syncthreads();
      const bool owner = (g == k + 1) && (k + 1 < n);   // column k+1 leaves its norm
      double sq = 0.0;
      for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
        const double vt = vs[t];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (g + q < j1) {
            double* p = W + (g + q) * s + k + t;
            const double val = fma(-wsum[q], vt, *p);
            *p = val;
            if (q == 0 && owner && t >= 1) sq = fma(val, val, sq);
          }
        }
      }
      if (owner) {
        sq = warp_sum(sq);
        if (lane == 0) nred[warp] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
          double q = 0.0;
          for (int w = 0; w < nw; ++w) q += nred[w];
          norms[k + 1] = q;
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, bar + 1, nb, err)) return;
  }
}

// FP64 variant with the columns resident in shared memory (s <= 4096 and at most
// kQr64sMaxCols columns per CTA), with look-ahead.  CTA b owns columns b, b + nb, ...
// (cyclic, so every CTA keeps a share of the trailing matrix to the end) and keeps them in
// shared memory for the whole factorization; each thread holds v_k for its rows in
// registers.  A CTA touches only its own columns, so steps need no grid barrier: step k
// waits (bounded) for the flag ready[k] that the owner of column k raises once column k
// (updated by reflectors 0..k-1) and its norm are in global memory.  The owner of column
// k+1 updates that column first, publishes it, then updates its other columns; the rest of
// the trailing update overlaps the next pivot's critical path.  ready[] (n + 1 words) must
// be zero at launch.  At the end the owner of column n (b) writes it back.
constexpr int kQr64sMaxCols = 8;
constexpr int kQr64sRows = 8;          // rows per thread: s <= 512 * 8

__device__ __forceinline__ double block_sum_512(double v, double* nred) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) nred[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int w = 0; w < nw; ++w) q += nred[w];
    nred[16] = q;
  }
  __syncthreads();
  return nred[16];
}

__global__ void __launch_bounds__(kQr64Threads, 1)
    qr64s_kernel(double* __restrict__ W, int64_t s, int64_t n, double* __restrict__ norms,
                 double* __restrict__ diagR, unsigned* __restrict__ ready, int* err) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  double* cols = reinterpret_cast<double*>(qr_smem);   // [owned][s]
  __shared__ double red[16 * 9];
  __shared__ double wsum[8];
  __shared__ double nred[17];
  __shared__ int ok_s;
  const int nb = (int)gridDim.x, b = (int)blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t ncols = n + 1;
  int owned = 0;
  for (int64_t j = b; j < ncols; j += nb) ++owned;
  for (int c = 0; c < owned; ++c) {
    const int64_t j = b + (int64_t)c * nb;
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) cols[c * s + t] = W[j * s + t];
  }
  __syncthreads();
  if (b == 0) {   // column 0 is ready as it stands: its norm, then the flag
    double part = 0.0;
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) part = fma(cols[t], cols[t], part);
    const double nn = block_sum_512(part, nred);
    if (threadIdx.x == 0) {
      norms[0] = nn;
      __threadfence();
      atomicExch(ready, 1u);
    }
  }
  for (int64_t k = 0; k < n; ++k) {
    // ---- wait for column k and its norm
    if (threadIdx.x == 0) {
      volatile unsigned* vr = ready + k;
      int ok = 1;
      if (*vr == 0u) {
        const uint64_t t0 = globaltimer_ns();
        while (*vr == 0u) {
          if (globaltimer_ns() - t0 > kWaitLimitNs) {
            set_error(err, DEV_TIMEOUT_GRID);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
      ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return;
    const double* colk = W + k * s;
    const double alpha = sqrt(__ldcg(norms + k));
    const double x0 = __ldcg(colk + k);
    const double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
    const double tau = (alpha > 0.0) ? 1.0 / (alpha * (alpha + fabs(x0))) : 0.0;
    if (b == 0 && threadIdx.x == 0) diagR[k] = -sgn * alpha;
    double v[kQr64sRows];
#pragma unroll
    for (int r = 0; r < kQr64sRows; ++r) {
      const int64_t t = threadIdx.x + (int64_t)r * blockDim.x;
      v[r] = (t < k || t >= s) ? 0.0 : (t == k ? x0 + sgn * alpha : __ldcg(colk + t));
    }
    // owned columns with index > k, from c_first on; the next pivot k+1 first if owned
    int c_first = 0;
    if (k + 1 > b) c_first = (int)((k + 1 - b + nb - 1) / nb);
    const int64_t jn = k + 1;
    if (jn < n && jn % nb == b) {
      const int cn = (int)(jn / nb);       // == c_first
      double d = 0.0;
#pragma unroll
      for (int r = 0; r < kQr64sRows; ++r) {
        const int64_t t = threadIdx.x + (int64_t)r * blockDim.x;
        if (t < s) d = fma(v[r], cols[cn * s + t], d);
      }
      const double wn = block_sum_512(d, nred) * tau;
      double sq = 0.0;
#pragma unroll
      for (int r = 0; r < kQr64sRows; ++r) {
        const int64_t t = threadIdx.x + (int64_t)r * blockDim.x;
        if (t < s && t >= k) {
          const double val = fma(-wn, v[r], cols[cn * s + t]);
          cols[cn * s + t] = val;
          if (t >= jn) sq = fma(val, val, sq);
        }
      }
      const double nn = block_sum_512(sq, nred);
      for (int64_t t = threadIdx.x; t < s; t += blockDim.x) W[jn * s + t] = cols[cn * s + t];
      __syncthreads();
      if (threadIdx.x == 0) {
        norms[jn] = nn;
        __threadfence();
        atomicExch(ready + jn, 1u);
      }
      c_first = cn + 1;
    }
    // ---- the other owned trailing columns, up to eight at a time
    if (c_first < owned) {
      double d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c_first + q;
        if (c < owned) {
#pragma unroll
          for (int r = 0; r < kQr64sRows; ++r) {
            const int64_t t = threadIdx.x + (int64_t)r * blockDim.x;
            if (t < s) d[q] = fma(v[r], cols[c * s + t], d[q]);
          }
        }
      }
      const double tot = warp_reduce8(d);
      if ((lane & 3) == 0) red[warp * 9 + ((lane >> 2) & 7)] = tot;
      __syncthreads();
      if (threadIdx.x < 8) {
        double q = 0.0;
        for (int w = 0; w < nw; ++w) q += red[w * 9 + threadIdx.x];
        wsum[threadIdx.x] = q * tau;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c_first + q;
        if (c < owned) {
          const double wq = wsum[q];
#pragma unroll
          for (int r = 0; r < kQr64sRows; ++r) {
            const int64_t t = threadIdx.x + (int64_t)r * blockDim.x;
            if (t < s && t >= k) cols[c * s + t] = fma(-wq, v[r], cols[c * s + t]);
          }
        }
      }
    }
    __syncthreads();
  }
  // columns 0..n-1 are final in W since they were published; only b's column is left
  if (n % nb == b) {
    const int c = (int)(n / nb);
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) W[n * s + t] = cols[c * s + t];
  }
}

// R (FP64, col-major, diag >= 0) and c from the factored work matrix.
template <typename T>
__device__ __forceinline__ void qr_finalize_body(const T* __restrict__ W, int64_t s, int64_t n,
                                                 const double* __restrict__ diagR, double* __restrict__ R,
                                                 double* __restrict__ c, int64_t j /* column of R */) {
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
__global__ void qr_finalize_kernel(const T* __restrict__ W, int64_t s, int64_t n,
                                   const double* __restrict__ diagR, double* __restrict__ R,
                                   double* __restrict__ c) {
  qr_finalize_body<T>(W, s, n, diagR, R, c, blockIdx.x);
}

// ------------------------------------------------------------ blocked variant
// Panels of NB columns: one CTA factors the panel W[p:s, p:p+kb] in shared
// memory (column Householder steps with block reductions), leaving the vectors
// v_j below the diagonal, tau_j = 1 / (alpha (alpha + |x_1|)) and the compact-WY
// factor T (Q_panel = I - V T V^T, T upper triangular, Schreiber-Van Loan
// recurrence); then every trailing column y (including the right-hand side) is
// updated as y -= V (T^T (V^T y)) by a grid of CTAs.  Same reflectors and the
// same arithmetic order per column as the unblocked kernel, blocked.
constexpr int kQrPanelThreads = 1024;

template <typename T>
__device__ __forceinline__ T block_sum_1024(T v, T* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T t = (threadIdx.x < 32) ? red[threadIdx.x] : T(0);
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  return red[32];
}

// Block-wide sums of NB per-thread values (entries c < lo are ignored).
template <typename T, int NB>
__device__ __forceinline__ void block_vsum(T (&pd)[NB], int lo, T (*red)[NB + 1], T* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c >= lo) {
      const T v = warp_sum(pd[c]);
      if (lane == 0) red[warp][c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < NB && (int)threadIdx.x >= lo) {
    T t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

template <typename T, int NB>
__global__ void __launch_bounds__(kQrPanelThreads)
    qr_panel_kernel(T* __restrict__ W, int64_t s, int64_t p, int kb, double* __restrict__ diagR,
                    T* __restrict__ tau, T* __restrict__ Tm) {
  extern __shared__ __align__(16) unsigned char qp_smem[];
  T* P = reinterpret_cast<T*>(qp_smem);        // [kb][len] panel, column-major
  __shared__ T red[32][NB + 1];
  __shared__ T wv[NB];
  __shared__ T tj_s;
  const int64_t len = s - p;
  for (int c = 0; c < kb; ++c)
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) P[c * len + t] = W[(p + c) * s + p + t];
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    T* x = P + j * len;
    T pd[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) pd[c] = 0;
    for (int64_t t = j + threadIdx.x; t < len; t += blockDim.x) pd[0] += x[t] * x[t];
    block_vsum<T, NB>(pd, 0, red, wv);
    if (threadIdx.x == 0) {
      const T alpha = sqrt(wv[0]);
      const T x0 = x[j];
      const T sgn = (x0 >= T(0)) ? T(1) : T(-1);
      const T tj = (alpha > T(0)) ? T(1) / (alpha * (alpha + fabs(x0))) : T(0);
      x[j] = x0 + sgn * alpha;               // v_j lives in rows j.. of panel column j
      diagR[p + j] = (double)(-sgn * alpha);
      tau[j] = tj;
      tj_s = tj;
    }
    __syncthreads();
    const T tj = tj_s;
    // w_c = tau_j v_j^T y_c for all remaining panel columns at once, then y_c -= w_c v_j
#pragma unroll
    for (int c = 0; c < NB; ++c) pd[c] = 0;
    for (int64_t t = j + threadIdx.x; t < len; t += blockDim.x) {
      const T xv = x[t];
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c > j && c < kb) pd[c] += xv * P[c * len + t];
    }
    block_vsum<T, NB>(pd, j + 1, red, wv);
    for (int64_t t = j + threadIdx.x; t < len; t += blockDim.x) {
      const T xv = x[t];
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c > j && c < kb) P[c * len + t] -= (wv[c] * tj) * xv;
    }
    __syncthreads();
  }
  // T factor: T_jj = tau_j ; T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j)
  if ((int)threadIdx.x < kb) Tm[threadIdx.x * NB + threadIdx.x] = tau[threadIdx.x];
  __syncthreads();
  for (int j = 1; j < kb; ++j) {
    const T* vj = P + j * len;
    T pd[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) pd[c] = 0;
    for (int64_t t = j + threadIdx.x; t < len; t += blockDim.x) {   // v_j is zero above row j
      const T vv = vj[t];
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < j) pd[c] += P[c * len + t] * vv;
    }
    block_vsum<T, NB>(pd, 0, red, wv);
    if (threadIdx.x == 0) {
      const T tjj = tau[j];
      for (int i = 0; i < j; ++i) {
        T acc = 0;
        for (int l = i; l < j; ++l) acc += Tm[l * NB + i] * wv[l];
        Tm[j * NB + i] = -tjj * acc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < NB) {
    const int j = threadIdx.x;
    for (int i = 0; i < NB; ++i)
      if (i > j || j >= kb) Tm[j * NB + i] = T(0);
  }
  // write back: rows 0..j-1 of column j are R entries, rows j.. hold v_j
  for (int c = 0; c < kb; ++c)
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) W[(p + c) * s + p + t] = P[c * len + t];
}

// y -= V T^T V^T y for trailing columns c in [p + kb, n] (column n = Omega b).
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    qr_trail_kernel(T* __restrict__ W, int64_t s, int64_t n, int64_t p, int kb,
                    const T* __restrict__ Tm) {
  __shared__ T red[NB][9];
  __shared__ T wv[NB];
  const int64_t len = s - p;
  const T* V = W + p * s + p;                  // column j of V at V + j * s (rows j.. are valid)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t col = p + kb + blockIdx.x; col <= n; col += gridDim.x) {
    T* y = W + col * s + p;
    // w = V^T y (v_j has an implicit zero above row j)
    for (int j = warp; j < kb; j += 8) {
      const T* vj = V + (int64_t)j * s;
      T pd = 0;
      for (int64_t t = j + lane; t < len; t += 32) pd += vj[t] * y[t];
      pd = warp_sum(pd);
      if (lane == 0) wv[j] = pd;
    }
    __syncthreads();
    // w2 = T^T w (T upper triangular): w2_j = sum_{i <= j} T(i, j) w_i
    if (threadIdx.x < kb) {
      const int j = threadIdx.x;
      T acc = 0;
      for (int i = 0; i <= j; ++i) acc += Tm[j * NB + i] * wv[i];
      red[j][0] = acc;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
      T acc = 0;
      const int jmax = (t < kb - 1) ? (int)t : kb - 1;
      for (int j = 0; j <= jmax; ++j) acc += V[(int64_t)j * s + t] * red[j][0];
      y[t] -= acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ register-panel variant
// The same blocked algorithm with the panel held in registers: 1024 threads,
// thread t owns panel rows t, t + 1024, ... (RPT rows), NB columns each.  A
// column costs two block reductions: ||x_j|| (with x_j[j] broadcast through
// shared memory so every thread forms alpha, tau and v_jj itself), then one
// reduction of v_j^T x_c for all other panel columns at once -- c > j are the
// update coefficients, c < j are the Gram entries v_c^T v_j from which warp 0
// extends the compact-WY factor T (T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j]).
// Within a warp the NB partial sums are reduced by recursive halving (NB
// shuffles instead of 5 NB).
constexpr int kQrRegThreads = 1024;

// After the call lane l holds the warp total of v[l >> 1] (N = 16).
template <int N>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[N], int lane) {
  static_assert(N == 16, "16 values over 32 lanes");
#pragma unroll
  for (int o = 16, cnt = N; o >= 2; o >>= 1, cnt >>= 1) {
    const bool upper = (lane & o) != 0;
    const int half = cnt / 2;
#pragma unroll
    for (int t = 0; t < N / 2; ++t) {
      if (t < half) {
        const float send = upper ? v[t] : v[t + half];
        const float keep = upper ? v[t + half] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int NB, int RPT>
__global__ void __launch_bounds__(kQrRegThreads, 1)
    qr_panel_reg_kernel(float* __restrict__ W, int64_t s, int64_t p, int kb, double* __restrict__ diagR,
                        float* __restrict__ tau, float* __restrict__ Tm) {
  __shared__ float redA[32];
  __shared__ float redB[32][NB];
  __shared__ float Ts[NB * NB];
  __shared__ float x0s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t len = s - p;
  float x[RPT][NB];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int64_t r = tid + (int64_t)i * kQrRegThreads;
#pragma unroll
    for (int c = 0; c < NB; ++c) x[i][c] = (r < len && c < kb) ? W[(p + c) * s + p + r] : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < kb) {
      // ---- alpha = ||x_j[j:]||, tau_j, v_jj
      float part = 0.0f;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int64_t r = tid + (int64_t)i * kQrRegThreads;
        if (r >= j) part += x[i][j] * x[i][j];
      }
      part = warp_sum(part);
      if (lane == 0) redA[warp] = part;
      if (tid == j) x0s = x[0][j];
      __syncthreads();
      const float n2 = warp_sum(redA[lane]);
      const float x0 = x0s;
      const float alpha = sqrtf(n2);
      const float sgn = (x0 >= 0.0f) ? 1.0f : -1.0f;
      const float tj = (alpha > 0.0f) ? 1.0f / (alpha * (alpha + fabsf(x0))) : 0.0f;
      if (tid == j) {
        x[0][j] = x0 + sgn * alpha;          // v_j lives in rows j.. of panel column j
        diagR[p + j] = (double)(-sgn * alpha);
        tau[j] = tj;
      }
      // ---- d_c = v_j^T x_c for every other column (rows >= j; v_j is zero above)
      float pw[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        pw[c] = 0.0f;
        if (c != j) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const int64_t r = tid + (int64_t)i * kQrRegThreads;
            if (r >= j) pw[c] += x[i][j] * x[i][c];
          }
        }
      }
      const float wsum = warp_reduce_scatter<NB>(pw, lane);
      if ((lane & 1) == 0) redB[warp][lane >> 1] = wsum;
      __syncthreads();
      float d = 0.0f;
      if (lane < NB) {
#pragma unroll 8
        for (int w = 0; w < 32; ++w) d += redB[w][lane];
      }
      // ---- trailing panel columns: x_c -= tau_j d_c v_j
#pragma unroll
      for (int c = j + 1; c < NB; ++c) {
        const float coef = tj * __shfl_sync(0xffffffffu, d, c);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int64_t r = tid + (int64_t)i * kQrRegThreads;
          if (r >= j) x[i][c] -= coef * x[i][j];
        }
      }
      // ---- T column j (warp 0): T_jj = tau_j, T[a, j] = -tau_j sum_{l=a}^{j-1} T[a, l] G[l, j]
      if (warp == 0) {
        float tcol = 0.0f;
#pragma unroll
        for (int l = 0; l < j; ++l) {
          const float g = __shfl_sync(0xffffffffu, d, l);
          if (lane <= l) tcol += Ts[lane + l * NB] * g;
        }
        if (lane < j) Ts[lane + j * NB] = -tj * tcol;
        if (lane == j) Ts[j + j * NB] = tj;
        if (lane > j && lane < NB) Ts[lane + j * NB] = 0.0f;
        __syncwarp();
      }
    } else if (warp == 0 && lane < NB) {
      Ts[lane + j * NB] = 0.0f;
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) Tm[e] = Ts[e];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int64_t r = tid + (int64_t)i * kQrRegThreads;
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (r < len && c < kb) W[(p + c) * s + p + r] = x[i][c];
  }
}

// y -= V T^T V^T y for the trailing columns (V in registers, one block
// reduction per column; reduction buffers alternate so one barrier suffices).
template <int NB, int RPT>
__global__ void __launch_bounds__(kQrRegThreads, 1)
    qr_trail_reg_kernel(float* __restrict__ W, int64_t s, int64_t n, int64_t p, int kb,
                        const float* __restrict__ Tm) {
  __shared__ float red[2][32][NB];
  __shared__ float Ts[NB * NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t len = s - p;
  for (int e = tid; e < NB * NB; e += blockDim.x) Ts[e] = Tm[e];
  float V[RPT][NB];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int64_t r = tid + (int64_t)i * kQrRegThreads;
#pragma unroll
    for (int c = 0; c < NB; ++c) V[i][c] = (r < len && c < kb && r >= c) ? W[(p + c) * s + p + r] : 0.0f;
  }
  __syncthreads();
  int par = 0;
  for (int64_t col = p + kb + blockIdx.x; col <= n; col += gridDim.x, par ^= 1) {
    float* y = W + col * s + p;
    float yv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int64_t r = tid + (int64_t)i * kQrRegThreads;
      yv[i] = (r < len) ? y[r] : 0.0f;
    }
    float pw[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      pw[c] = 0.0f;
#pragma unroll
      for (int i = 0; i < RPT; ++i) pw[c] += V[i][c] * yv[i];
    }
    const float wsum = warp_reduce_scatter<NB>(pw, lane);
    if ((lane & 1) == 0) red[par][warp][lane >> 1] = wsum;
    __syncthreads();
    float w = 0.0f;
    if (lane < NB) {
#pragma unroll 8
      for (int q = 0; q < 32; ++q) w += red[par][q][lane];
    }
    // w2 = T^T w: w2_c = sum_{a <= c} T[a, c] w_a
    float w2 = 0.0f;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const float wa = __shfl_sync(0xffffffffu, w, a);
      if (lane < NB && a <= lane) w2 += Ts[a + lane * NB] * wa;
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const float w2c = __shfl_sync(0xffffffffu, w2, c);
#pragma unroll
      for (int i = 0; i < RPT; ++i) yv[i] -= V[i][c] * w2c;
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int64_t r = tid + (int64_t)i * kQrRegThreads;
      if (r < len) y[r] = yv[i];
    }
  }
}

template <int RPT>
static cudaError_t run_qr_reg(const double* Y, int64_t s, int64_t n, float* W, double* aux, double* R,
                              double* c, int num_sms, cudaStream_t st) {
  constexpr int NB = 16;
  const int64_t total = s * (n + 1);
  convert_y_kernel<float><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Y, W, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* diagR = aux + n;
  float* tau = reinterpret_cast<float*>(aux + 2 * n + 8);
  float* Tm = tau + NB;
  for (int64_t p = 0; p < n; p += NB) {
    const int kb = (int)std::min<int64_t>(NB, n - p);
    qr_panel_reg_kernel<NB, RPT><<<1, kQrRegThreads, 0, st>>>(W, s, p, kb, diagR, tau, Tm);
    const int64_t ncols = n + 1 - (p + kb);
    if (ncols > 0) {
      const unsigned grid = (unsigned)std::min<int64_t>(ncols, (int64_t)num_sms);
      qr_trail_reg_kernel<NB, RPT><<<grid, kQrRegThreads, 0, st>>>(W, s, n, p, kb, Tm);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qr_finalize_kernel<float><<<(unsigned)n, 256, 0, st>>>(W, s, n, diagR, R, c);
  return cudaGetLastError();
}

template <typename T>
static bool qr_blocked_fits(int64_t s, int nb) {
  return (size_t)s * nb * sizeof(T) <= 200 * 1024;
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
    e = allow_dyn_smem(kern, smem);
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

static cudaError_t run_qr64(const double* Y, int64_t s, int64_t n, double* W, double* aux, unsigned* bar,
                           double* R, double* c, int* err, int num_sms, cudaStream_t st) {
  const int64_t total = s * (n + 1);
  cudaError_t e = cudaMemcpyAsync(W, Y, (size_t)total * 8, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int grid = num_sms;                      // one CTA per SM (co-resident: occ >= 1)
  const int64_t per_cta = (n + 1 + grid - 1) / grid;
  const bool resident = s <= (int64_t)kQr64Threads * kQr64sRows && per_cta <= kQr64sMaxCols &&
                        (size_t)per_cta * s * 8 <= 227 * 1024 - 2048;
  auto kern = resident ? qr64s_kernel : qr64_kernel;
  const size_t smem = resident ? (size_t)per_cta * s * 8 : (size_t)s * 8;
  e = allow_dyn_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kQr64Threads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  double* norms = aux;
  double* diagR = aux + n;
  // the resident kernel's per-column flags follow diag(R) in aux (n + 1 words, zeroed here)
  unsigned* ready = reinterpret_cast<unsigned*>(aux + 2 * n + 8);
  if (resident) {
    e = cudaMemsetAsync(ready, 0, (size_t)(n + 1) * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  unsigned* sync = resident ? ready : bar;
  double* Wp = W;
  int64_t sp = s, np = n;
  void* args[] = {&Wp, &sp, &np, &norms, &diagR, &sync, &err};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(kQr64Threads), args, smem, st);
  if (e != cudaSuccess) return e;
  qr_finalize_kernel<double><<<(unsigned)n, 256, 0, st>>>(W, s, n, diagR, R, c);
  return cudaGetLastError();
}

template <typename T, int NB>
static cudaError_t run_qr_blocked(const double* Y, int64_t s, int64_t n, T* W, double* aux, double* R,
                                  double* c, int num_sms, cudaStream_t st) {
  const int64_t total = s * (n + 1);
  convert_y_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Y, W, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* diagR = aux + n;
  T* tau = reinterpret_cast<T*>(aux + 2 * n + 8);
  T* Tm = tau + NB;
  const size_t smem = (size_t)s * NB * sizeof(T);
  e = allow_dyn_smem(qr_panel_kernel<T, NB>, smem);
  if (e != cudaSuccess) return e;
  for (int64_t p = 0; p < n; p += NB) {
    const int kb = (int)std::min<int64_t>(NB, n - p);
    qr_panel_kernel<T, NB><<<1, kQrPanelThreads, (size_t)(s - p) * kb * sizeof(T), st>>>(W, s, p, kb, diagR,
                                                                                        tau, Tm);
    const int64_t ncols = n + 1 - (p + kb);
    if (ncols > 0) {
      const unsigned grid = (unsigned)std::min<int64_t>(ncols, 4 * (int64_t)num_sms);
      qr_trail_kernel<T, NB><<<grid, 256, 0, st>>>(W, s, n, p, kb, Tm);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qr_finalize_kernel<T><<<(unsigned)n, 256, 0, st>>>(W, s, n, diagR, R, c);
  return cudaGetLastError();
}

cudaError_t launch_qr(bool fp64, const double* Y, int64_t s, int64_t n, void* work, double* aux,
                      unsigned* bar, double* R, double* c, int* err, int num_sms, cudaStream_t st) {
  if (!fp64 && s <= kQrRegThreads)
    return run_qr_reg<1>(Y, s, n, static_cast<float*>(work), aux, R, c, num_sms, st);
  if (!fp64 && s <= 2 * kQrRegThreads)
    return run_qr_reg<2>(Y, s, n, static_cast<float*>(work), aux, R, c, num_sms, st);
  if (!fp64 && qr_blocked_fits<float>(s, 24))
    return run_qr_blocked<float, 24>(Y, s, n, static_cast<float*>(work), aux, R, c, num_sms, st);
  if (fp64)
    return run_qr64(Y, s, n, static_cast<double*>(work), aux, bar, R, c, err, num_sms, st);
  return run_qr<float>(Y, s, n, static_cast<float*>(work), aux, bar, R, c, err, num_sms, st);
}


// ============================================================ grouped (batched) QR
// One 1024-thread CTA per problem (s <= 1024): the reflectors of qr_kernel, v in shared
// memory, whole trailing columns per warp (lanes over rows, one warp sum per dot
// product); the warp that updates column k+1 also sums its squares below the diagonal
// for the next step's norm.  W (s x (n + 1), ld = s) stays in global memory.
template <typename T>
__global__ void __launch_bounds__(1024) grouped_qr_kernel(const GQr<T>* __restrict__ tab) {
  const GQr<T>& g = tab[blockIdx.x];
  const int64_t s = g.s, n = g.n;
  T* W = g.W;
  __shared__ T vs[1024];
  __shared__ T red[33];
  __shared__ T nrm_next;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t e = threadIdx.x; e < s * (n + 1); e += blockDim.x) W[e] = (T)g.Y[e];
  __syncthreads();
  T part = 0;
  for (int64_t t = threadIdx.x; t < s; t += blockDim.x) part += W[t] * W[t];
  T nn = block_sum_1024(part, red);
  for (int64_t k = 0; k < n; ++k) {
    const T* colk = W + k * s;
    const T alpha = sqrt(nn);
    const T x0 = colk[k];
    const T sgn = (x0 >= T(0)) ? T(1) : T(-1);
    const T scale = (alpha > T(0)) ? T(1) / (alpha * (alpha + fabs(x0))) : T(0);
    if (threadIdx.x == 0) g.diagR[k] = (double)(-sgn * alpha);
    const int64_t len = s - k;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) vs[t] = (t == 0) ? x0 + sgn * alpha : colk[k + t];
    __syncthreads();
    for (int64_t j = k + 1 + warp; j <= n; j += nw) {
      T* colj = W + j * s + k;
      T d = 0;
      for (int64_t t = lane; t < len; t += 32) d += vs[t] * colj[t];
      const T wj = warp_sum(d) * scale;
      T sq = 0;
      for (int64_t t = lane; t < len; t += 32) {
        const T val = colj[t] - wj * vs[t];
        colj[t] = val;
        if (t >= 1) sq += val * val;
      }
      if (j == k + 1) {
        sq = warp_sum(sq);
        if (lane == 0) nrm_next = sq;
      }
    }
    __syncthreads();
    nn = nrm_next;
  }
}

template <typename T>
__global__ void grouped_qr_finalize_kernel(const GQr<T>* __restrict__ tab, const int* __restrict__ start, int nprob) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GQr<T>& g = tab[p];
  qr_finalize_body<T>(g.W, g.s, g.n, g.diagR, g.R, g.c, (int64_t)blockIdx.x - start[p]);
}

template <typename T>
cudaError_t launch_grouped_qr(const GQr<T>* tab, const int* col_start, int64_t col_ctas, int nprob, int64_t max_n,
                              cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  (void)max_n;
  grouped_qr_kernel<T><<<(unsigned)nprob, 1024, 0, st>>>(tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grouped_qr_finalize_kernel<T><<<(unsigned)col_ctas, 256, 0, st>>>(tab, col_start, nprob);
  return cudaGetLastError();
}
template cudaError_t launch_grouped_qr<float>(const GQr<float>*, const int*, int64_t, int, int64_t, cudaStream_t);
template cudaError_t launch_grouped_qr<double>(const GQr<double>*, const int*, int64_t, int, int64_t, cudaStream_t);

}  // namespace lsq
