// Double-double (u ~ 2^-106) products of Algorithm 2 for u = double:
//   * the refinement residual [f; g] = [b - r - A x; -A^T r] in u_r = double-double,
//   * the FGMRES products of the Sec. 5 escalation (u_A = u_L = u_R = quad when u is
//     double): z = R^-1 v_bot, w_top = alpha v_top + A z, w_bot = R^-T (A^T v_top).
// A and R are FP64; every product is split exactly (TwoProduct) and summed in
// double-double, and each result is rounded once to FP64 where the method stores it
// (the Krylov basis and the residual vectors are FP64).  These run on the FP64 pipe,
// about a dozen FP64 operations per matrix entry: they are the accuracy path of u =
// double, not a bandwidth-bound pass.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "dd.cuh"
#include "iter.h"

namespace lsq {

namespace {

constexpr int kDdRowsThreads = 256;
constexpr int kDdTrsvThreads = 1024;
constexpr int kDdTrsvMaxN = 1024;

struct DdRowsArgs {
  const double* A;
  int64_t lda, m, n;
  const double* zh;
  const double* zl;
  int64_t zstr;
  const double* u;
  double cu;
  int64_t ustr;
  const double* w;
  double cw;
  double sgn;
  double* out;
  const int* done;
  const int* jp;
};

// out[i] = fl(cu u[i] + cw w[i] + sgn sum_k A[i][k] (zh[k] + zl[k])): one warp per row,
// lanes over the columns, a butterfly sum of the lanes' double-double partials.
__global__ void __launch_bounds__(kDdRowsThreads) dd_rows_kernel(const DdRowsArgs a) {
  if (a.done && *a.done) return;
  const int64_t jc = a.jp ? *a.jp : 0;
  const double* zh = a.zh + jc * a.zstr;
  const double* zl = a.zl;
  const double* u = a.u ? a.u + jc * a.ustr : nullptr;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < a.m; i += nw) {
    const double* Ai = a.A + i * a.lda;
    DD acc{0.0, 0.0};
    for (int64_t k = lane; k < a.n; k += 32) acc = dd_fma(acc, Ai[k], zh[k], zl ? zl[k] : 0.0);
    acc = dd_warp_sum(acc);
    if (lane == 0) {
      if (a.sgn < 0.0) {
        acc.hi = -acc.hi;
        acc.lo = -acc.lo;
      }
      DD p;
      if (u) {
        two_prod(a.cu, u[i], p.hi, p.lo);
        acc = dd_add(acc, p);
      }
      if (a.w) {
        two_prod(a.cw, a.w[i], p.hi, p.lo);
        acc = dd_add(acc, p);
      }
      a.out[i] = __dadd_rn(acc.hi, acc.lo);
    }
  }
}

// P[blk][k] = sum over the block's rows of A[i][k] v[i] (double-double, hi and lo planes):
// 32 columns x 8 row phases per CTA, the eight phase sums added in a fixed order.
__global__ void __launch_bounds__(256) dd_cols_kernel(const double* __restrict__ A, int64_t lda, int64_t m,
                                                      int64_t n, const double* __restrict__ v, int64_t vstr,
                                                      double* Phi, double* Plo, const int* done,
                                                      const int* jp) {
  if (done && *done) return;
  __shared__ double sh[8][33], sl[8][33];
  const int64_t jc = jp ? *jp : 0;
  const double* vv = v + jc * vstr;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t chunk = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(m, r0 + chunk);
  for (int64_t c0 = 0; c0 < n; c0 += 32) {
    const int64_t col = c0 + tx;
    DD acc{0.0, 0.0};
    if (col < n)
      for (int64_t i = r0 + ty; i < r1; i += 8) acc = dd_fma(acc, A[i * lda + col], vv[i], 0.0);
    sh[ty][tx] = acc.hi;
    sl[ty][tx] = acc.lo;
    __syncthreads();
    if (ty == 0 && col < n) {
      DD t{sh[0][tx], sl[0][tx]};
      for (int q = 1; q < 8; ++q) t = dd_add(t, DD{sh[q][tx], sl[q][tx]});
      Phi[(int64_t)blockIdx.x * n + col] = t.hi;
      Plo[(int64_t)blockIdx.x * n + col] = t.lo;
    }
    __syncthreads();
  }
}

// out[k] = sgn sum_blk P[blk][k] in block order (double-double); out_lo may be null
// (then out_hi holds the value rounded to FP64).
__global__ void dd_colsum_kernel(const double* __restrict__ Phi, const double* __restrict__ Plo, int nblk,
                                 int64_t n, double sgn, double* out_hi, double* out_lo, const int* done) {
  if (done && *done) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  DD t{0.0, 0.0};
  for (int b = 0; b < nblk; ++b) t = dd_add(t, DD{Phi[(int64_t)b * n + k], Plo[(int64_t)b * n + k]});
  if (sgn < 0.0) {
    t.hi = -t.hi;
    t.lo = -t.lo;
  }
  if (out_lo) {
    out_hi[k] = t.hi;
    out_lo[k] = t.lo;
  } else {
    out_hi[k] = __dadd_rn(t.hi, t.lo);
  }
}

// x = R^-1 y (upper) or R^-T y (lower) in double-double, one CTA.  Blocks of 32
// unknowns: warp 0 solves the diagonal block (lane l holds unknown j0 + l; the owner of
// unknown j divides and broadcasts it, lanes of the later unknowns take its product off),
// then every thread takes the block's 32 products off one remaining row.  R64 holds
// R(i, j) at j ld + i and L64 holds R(i, j) at i ld + j, so both updates read
// consecutive addresses across threads.
__global__ void __launch_bounds__(kDdTrsvThreads)
    dd_trsv_kernel(bool upper, const double* __restrict__ R64, const double* __restrict__ L64, int64_t ld,
                   int n, const double* in_hi, const double* in_lo, int64_t in_str, double* out_hi,
                   int64_t out_str, double* out_lo, const int* done, const int* jp) {
  if (done && *done) return;
  __shared__ double xh[kDdTrsvMaxN], xl[kDdTrsvMaxN];
  __shared__ double zh[32], zl[32];
  const int64_t jc = jp ? *jp : 0;
  const double* yh = in_hi + jc * in_str;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xh[i] = yh[i];
    xl[i] = in_lo ? in_lo[i] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (n + 31) / 32;
  for (int q = 0; q < nb; ++q) {
    const int blk = upper ? nb - 1 - q : q;
    const int j0 = blk * 32, j1 = min(n, j0 + 32), len = j1 - j0;
    if (warp == 0) {
      DD xv{0.0, 0.0};
      if (lane < len) xv = DD{xh[j0 + lane], xl[j0 + lane]};
      for (int s = 0; s < len; ++s) {
        const int t = upper ? len - 1 - s : s;   // local index of the unknown solved now
        const int j = j0 + t;
        DD z{0.0, 0.0};
        if (lane == t) z = dd_div_d(xv, R64[(int64_t)j * ld + j]);
        z.hi = __shfl_sync(0xffffffffu, z.hi, t);
        z.lo = __shfl_sync(0xffffffffu, z.lo, t);
        if (lane == t) {
          xv = z;
        } else if (upper ? (lane < t) : (lane > t && lane < len)) {
          // upper: R(j0 + lane, j) z_j; lower: R^T(j0 + lane, j) z_j = R(j, j0 + lane) z_j
          const double rij = upper ? R64[(int64_t)j * ld + j0 + lane] : L64[(int64_t)j * ld + j0 + lane];
          xv = dd_fma(xv, -rij, z.hi, z.lo);
        }
      }
      if (lane < len) {
        xh[j0 + lane] = xv.hi;
        xl[j0 + lane] = xv.lo;
        zh[lane] = xv.hi;
        zl[lane] = xv.lo;
      }
    }
    __syncthreads();
    // remaining rows: upper, i < j0 (x_i -= R(i, j) z_j); lower, i >= j1 (x_i -= R(j, i) z_j)
    const int r0 = upper ? 0 : j1, r1 = upper ? j0 : n;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      DD acc{xh[i], xl[i]};
      for (int t = 0; t < len; ++t) {
        const int j = j0 + t;
        const double rij = upper ? R64[(int64_t)j * ld + i] : L64[(int64_t)j * ld + i];
        acc = dd_fma(acc, -rij, zh[t], zl[t]);
      }
      xh[i] = acc.hi;
      xl[i] = acc.lo;
    }
    __syncthreads();
  }
  double* oh = out_hi + jc * out_str;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (out_lo) {
      oh[i] = xh[i];
      out_lo[i] = xl[i];
    } else {
      oh[i] = __dadd_rn(xh[i], xl[i]);
    }
  }
}

}  // namespace

cudaError_t launch_dd_rows(const double* A, int64_t lda, int64_t m, int64_t n, const double* zh,
                           const double* zl, int64_t zstr, const double* u, double cu, int64_t ustr,
                           const double* w, double cw, double sgn, double* out, const int* done, const int* jp,
                           int num_sms, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  DdRowsArgs a{A, lda, m, n, zh, zl, zstr, u, cu, ustr, w, cw, sgn, out, done, jp};
  const int64_t warps = m < (int64_t)num_sms * 64 ? m : (int64_t)num_sms * 64;
  const unsigned grid = (unsigned)((warps * 32 + kDdRowsThreads - 1) / kDdRowsThreads);
  dd_rows_kernel<<<grid, kDdRowsThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dd_cols(const double* A, int64_t lda, int64_t m, int64_t n, const double* v, int64_t vstr,
                           double* Phi, double* Plo, int nblk, const int* done, const int* jp, cudaStream_t st) {
  if (nblk < 1) return cudaErrorInvalidValue;
  dd_cols_kernel<<<(unsigned)nblk, 256, 0, st>>>(A, lda, m, n, v, vstr, Phi, Plo, done, jp);
  return cudaGetLastError();
}

cudaError_t launch_dd_colsum(const double* Phi, const double* Plo, int nblk, int64_t n, double sgn,
                             double* out_hi, double* out_lo, const int* done, cudaStream_t st) {
  dd_colsum_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(Phi, Plo, nblk, n, sgn, out_hi, out_lo, done);
  return cudaGetLastError();
}

cudaError_t launch_dd_trsv(bool upper, const Tri<double>& f, const double* in_hi, const double* in_lo,
                           int64_t in_str, double* out_hi, int64_t out_str, double* out_lo, const int* done,
                           const int* jp, cudaStream_t st) {
  if (f.n > kDdTrsvMaxN || f.n < 1) return cudaErrorInvalidValue;
  dd_trsv_kernel<<<1, kDdTrsvThreads, 0, st>>>(upper, f.R, f.L, f.ld, (int)f.n, in_hi, in_lo, in_str, out_hi,
                                               out_str, out_lo, done, jp);
  return cudaGetLastError();
}

}  // namespace lsq
