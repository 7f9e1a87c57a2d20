// Grouped (batched) launches: one launch per stage for a batch of problems of uneven
// size.  Problem p owns the CTAs [start[p], start[p + 1]) of a grouped launch (start:
// nprob + 1 prefix sums built by the host), and each CTA reads its problem's arguments
// from a device table indexed by p.  Every per-problem computation is the one the
// single-problem kernels do, on the same blocking of that problem, so a problem's result
// does not depend on the other problems of the batch.  A problem whose state is done
// (LSQR converged, FGMRES converged, refinement finished) is skipped by its CTAs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "iter.h"
#include "kernels.h"

namespace lsq {

constexpr int kMaxGmresBatch = 80;   // FGMRES cap per refinement step in batched mode

template <typename TP, typename TO>
struct GColsum {
  const TP* P;
  int nblk;
  int64_t n;
  const double* scale_ptr;
  double scale_mul;
  TO* out;
  const int* done;
};

template <typename TP>
struct GLsqrColsum {
  const TP* P;
  int nblk;
  int64_t n;
  const double* sq;
  LsqrState* st;
  TP* out;
};

template <typename T>
struct GLsqrStep {
  Tri<T> f;
  const T* s;
  T* v;
  T* w;
  T* z;
  T* t;
  LsqrState* st;
};

template <typename TX, typename TY, typename TO>
struct GAxpby {
  const TX* x;
  double a;
  const TY* y;
  double b;
  TO* out;
  int64_t len;
  const int* done;
};

// x = M^-1 (yscale y) (one CTA per problem, n <= 1024), as launch_trsv's single-CTA solver.
template <typename T, typename TIN, typename TOUT>
struct GTrsv {
  const T* M;
  const T* D;
  int64_t ld;
  int n;
  const TIN* y;
  double yscale;
  TOUT* x;
  const int* done;
  const int* jp;
  int64_t ys, xstr;
};

struct GNorm {
  const double* x;
  int64_t len;
  double* out;   // ||x||
};

// FGMRES of one problem: the state, basis and work vectors of Alg. 2 (FGMRES solve).
struct GGm {
  double* V;            // (m + n) x (maxc), ld = m + n
  int64_t ld, m, n;
  double* w;            // work vector, m + n
  const void* az;       // A z left by the pass (FP32 or FP64), or null (w_top formed)
  int az_f32;
  GmState* st;
  int maxc, ldh;
  double* Dp;           // partials, [maxc + 1][nb]
  double* hs1;          // first Gram-Schmidt pass: h_0..h_j and ||w||^2 (maxc + 2)
  double* hs2;          // second pass
  double* H;
  double* cs;
  double* sn;
  double* g;
  double* y;
  float* v32;           // FP32 copy of the new column's top part (FP32 passes), or null
  double alpha;         // Sec. 4.1 scaling
  const double* f;      // right-hand side [f; h]
  const double* h;
  double* sqp;          // per-CTA partials of ||[f; h/alpha]||^2
  const int* skip;      // refinement mask: the problem takes no FGMRES solve when *skip
  const void* Zb;       // preconditioned vectors z_j (FP32 or FP64), ld = ldz
  int zb_f32;
  int64_t ldz;
  double* r;
  double* x;
  double* p4;           // 4 x nb partials of the update
  double* nrm;          // ||dr||^2, ||r||^2, ||dx||^2, ||x||^2
};

// ---- k_iter.cu
// the register-blocked pass over A for every problem (vw: vector width, vpl: vectors per
// lane, covering every problem's row; smem: 8 x (the widest row) x sizeof(T)).  ctas items
// (start[nprob]); grid: CTAs of the persistent launch (0 or >= ctas: one per item); the
// result is the same for every grid.
template <typename T>
cudaError_t launch_grouped_pass(int mode, int vw, int vpl, const PassArgs<T>* tab, const int* start,
                                int64_t ctas, int nprob, size_t smem, cudaStream_t st, int64_t grid = 0);
template <typename TP, typename TO>
cudaError_t launch_grouped_colsum(const GColsum<TP, TO>* tab, const int* start, int64_t ctas, int nprob,
                                  cudaStream_t st);
template <typename TP>
cudaError_t launch_grouped_lsqr_colsum(const GLsqrColsum<TP>* tab, const int* start, int64_t ctas, int nprob,
                                       bool init, cudaStream_t st);
template <typename T>
cudaError_t launch_grouped_lsqr_step(const GLsqrStep<T>* tab, int nprob, bool init, cudaStream_t st);
template <typename TX, typename TY, typename TO>
cudaError_t launch_grouped_axpby(const GAxpby<TX, TY, TO>* tab, const int* start, int64_t ctas, int nprob,
                                 cudaStream_t st);
cudaError_t launch_grouped_norm(const GNorm* tab, int nprob, cudaStream_t st);
// FGMRES: rhs and first column (start: Arnoldi CTAs per problem)
cudaError_t launch_grouped_gm_init(const GGm* tab, const int* start, int64_t ctas, int nprob, cudaStream_t st);
// one Arnoldi step (classical Gram-Schmidt, second pass where the first lost more than
// half of ||w||^2, new column, Givens step), in five to eight launches, no grid-wide waits
cudaError_t launch_grouped_arnoldi(const GGm* tab, const int* start, int64_t ctas, int nprob, cudaStream_t st);
// y = H^-1 g, r += alpha V_top y, x += Z y, and the four norms
cudaError_t launch_grouped_gm_update(const GGm* tab, const int* start, int64_t ctas, int nprob,
                                     cudaStream_t st);

// ---- k_trsv.cu
template <typename T, typename TIN, typename TOUT>
cudaError_t launch_grouped_trsv(bool upper, const GTrsv<T, TIN, TOUT>* tab, int nprob, cudaStream_t st);
// R copies of every problem (as launch_prepare_r): Rtab[p] = {R (n x n, FP64), n}; grids of n_p columns
struct GPrepR {
  const double* R;
  int64_t n;
  Tri<float> f32;
  Tri<double> f64;
  double* kappa;
};
cudaError_t launch_grouped_prepare_r(const GPrepR* tab, const int* col_start, int64_t col_ctas,
                                     const int* blk_start, int64_t blk_ctas, int nprob, cudaStream_t st);

// ---- k_qr.cu: Householder QR of each problem's sketch, one CTA per problem (s <= 1024)
template <typename T>
struct GQr {
  const double* Y;   // s x (n + 1), column-major
  T* W;              // work copy
  int64_t s, n;
  double* diagR;     // n
  double* R;         // n x n, column-major, diag >= 0
  double* c;         // n: (Q^T Omega b)[:n]
};
template <typename T>
cudaError_t launch_grouped_qr(const GQr<T>* tab, const int* col_start, int64_t col_ctas, int nprob, int64_t max_n,
                              cudaStream_t st);

}  // namespace lsq
