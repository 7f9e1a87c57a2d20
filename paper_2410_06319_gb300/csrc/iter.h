// Device-resident state of the iterative stages and the launch wrappers of
// their small kernels (LSQR, FGMRES, vector reductions).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace lsq {

// Arguments of the register-blocked pass over A (one problem):
//   PM_LSQR: q = A x + cu u_in ; u_out = q ; Pblk = A^T q per CTA ; sq = sum q^2 per CTA
//   PM_FGM : az = A x ; Pblk = A^T v
//   PM_RES : f = b - r - A x ; Pblk = A^T (-r)
enum PassMode { PM_LSQR = 0, PM_FGM = 1, PM_RES = 2 };

template <typename T>
struct PassArgs {
  const T* A;
  int64_t lda, m;
  int n, nv;             // nv = vectors per row (ceil(n / VW), padded rows for A32)
  const T* x;            // multiplied vector, nv * VW entries (zero padded)
  const T* uin;          // LSQR
  T* uout;
  const double* cu_ptr;
  double cu_mul;
  const T* v;            // FGMRES coefficient vector
  T* az;                 // FGMRES: A x
  const double* r;       // residual
  const double* b;
  double* f;
  T* Pblk;
  double* sq;
  const int* done;
  const int* jp;         // FGMRES: x and v are column (*jp) of their bases
  int64_t xstr, vstr;
};

// LSQR (Paige & Saunders 1982) scalars, kept on the device so that iterations
// run without host round trips; kernels of an iteration exit early once done.
struct LsqrState {
  double alpha, beta, rhobar, phibar, anorm2, normb, tol;
  double normr, normar, normA;
  double us;   // u = u_stored * us (u_stored is the unnormalised q)
  double cu;   // coefficient of u_stored in the next pass: -alpha * us
  int its, flag, done, maxit;
};

// FGMRES scalars (Arnoldi column count j, residual estimate).
struct GmState {
  double beta0, relres, tol, inv_h;
  int j, done, maxit, pad;
  int reorth;     // 1: the current Arnoldi step needs the second Gram-Schmidt pass
  int nreorth;    // second passes run so far
};

// LSQR pass over A (FP32 copy or FP64): q_i = (A t)_i + cu * u_i (cu read from *cu_ptr
// times cu_mul); u_out = q; Pblk[blk][c] = sum_rows q_i A_ic; sq[blk] = sum q_i^2.
template <typename TP>
cudaError_t launch_pass_lsqr_any(const TP* A, int64_t lda, int64_t m, int64_t n, const TP* t,
                                 const TP* u_in, const double* cu_ptr, double cu_mul, TP* u_out,
                                 TP* Pblk, double* sq, int nblk, const int* done, cudaStream_t st);
template <typename T>
cudaError_t launch_lsqr_colsum(const T* P, int nblk, int64_t n, const double* sq, LsqrState* st,
                               bool init, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_lsqr_step(const Tri<T>& f, const T* s, T* v, T* w, T* z, T* t, LsqrState* st,
                             bool init, cudaStream_t strm);

template <typename TX, typename TY, typename TO>
cudaError_t launch_axpby(const TX* x, double a, const TY* y, double b, TO* out, int64_t len,
                         cudaStream_t st);
cudaError_t launch_dot(const double* x, const double* y, int64_t len, double* partial, int nblk,
                       double* out, bool take_sqrt, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partial, int nblk, double* out, bool take_sqrt,
                                cudaStream_t st);

// V0 = [f; h / alpha] (alpha scales the augmented system, Sec. 4.1; 1 for the unscaled one)
cudaError_t launch_gm_rhs(const double* f, const double* h, int64_t m, int64_t n, double* V0,
                          double* sq_partial, int nblk, cudaStream_t s, double alpha = 1.0);
cudaError_t launch_gm_init(const double* sq_partial, int nblk, GmState* st, double* g, cudaStream_t s);
cudaError_t launch_gm_scale0(double* V0, int64_t len, const GmState* st, float* v32, int64_t m,
                             int nblk, cudaStream_t s);
// The whole Arnoldi step in one cooperative launch (gs = 0: classical Gram-Schmidt with the
// twice-is-enough second pass; 1: modified Gram-Schmidt, w in shared memory where it fits;
// 2: modified, w in global memory -- its grid sums use the 64-bit arrival counter *seq,
// zero before the solve's first step, every step of a solve on the same grid; Givens step,
// new column;
// blocks synchronised by a bounded last-arrival reduction on bar[0..1], which must be zero
// before the first launch; each launch leaves it reusable).  Dp holds (maxc + 1) x 2
// num_sms doubles; maxc <= 128.  Each sync waits at most wait_ns (0: the library's
// limit); a wait that runs out records DEV_TIMEOUT_GRID in *err and sets st->done, so the
// rest of the batch is skipped.
template <typename TAZ>
cudaError_t launch_gm_step(double* V, int64_t ld, double* w, int64_t len, int64_t m, const TAZ* az,
                           GmState* st, int maxc, double* Dp, double* sq, double* hsum, double* H, int ldh,
                           double* cs, double* sn, double* g, float* v32, unsigned* bar, int* err,
                           int num_sms, cudaStream_t s, uint64_t wait_ns = 0, double alpha = 1.0,
                           int gs = 0, unsigned long long* seq = nullptr, int expire = 0);
// modified Gram-Schmidt from this many rows of [r; x] on (opts.arnoldi = 0)
constexpr int64_t kMgsMinRows = (int64_t)3 << 18;   // 786,432: measured crossover ~7e5 on GB300
cudaError_t launch_gm_solve(const GmState* st, const double* H, int ldh, const double* g, double* y,
                            cudaStream_t s);
// d += scale (B y) over the first st->j columns of B; partial sums of ||scale B y||^2 and ||d||^2
template <typename TB>
cudaError_t launch_gm_apply(const TB* B, int64_t ld, int64_t len, const GmState* st, const double* y,
                            double* d, double* part_dd, double* part_d, int nblk, cudaStream_t s,
                            double scale = 1.0);

// ---- double-double products (u_r = double-double; u_A = u_L = u_R = quad for u double)
// out[i] = fl(cu u[i] + cw w[i] + sgn sum_k A[i][k] (zh[k] + zl[k])), i < m.  With jp, zh and u
// are offset by (*jp) * zstr and (*jp) * ustr; u, w and zl may be null.  Skips when *done.
cudaError_t launch_dd_rows(const double* A, int64_t lda, int64_t m, int64_t n, const double* zh,
                           const double* zl, int64_t zstr, const double* u, double cu, int64_t ustr,
                           const double* w, double cw, double sgn, double* out, const int* done, const int* jp,
                           int num_sms, cudaStream_t st);
// Phi/Plo[blk][k] = double-double partial of sum_i A[i][k] v[i] over the rows of block blk
// (nblk blocks); v offset by (*jp) * vstr.
cudaError_t launch_dd_cols(const double* A, int64_t lda, int64_t m, int64_t n, const double* v, int64_t vstr,
                           double* Phi, double* Plo, int nblk, const int* done, const int* jp, cudaStream_t st);
// out = sgn sum_blk P[blk] as double-double (out_lo != null) or rounded to FP64
cudaError_t launch_dd_colsum(const double* Phi, const double* Plo, int nblk, int64_t n, double sgn,
                             double* out_hi, double* out_lo, const int* done, cudaStream_t st);
// x = R^-1 y (upper) or R^-T y in double-double (n <= 1024, one CTA); y = in_hi (+ in_lo),
// in_hi offset by (*jp) * in_str and out_hi by (*jp) * out_str; out_lo null: out_hi holds
// x rounded to FP64, else x = out_hi + out_lo.
cudaError_t launch_dd_trsv(bool upper, const Tri<double>& f, const double* in_hi, const double* in_lo,
                           int64_t in_str, double* out_hi, int64_t out_str, double* out_lo, const int* done,
                           const int* jp, cudaStream_t st);

}  // namespace lsq
