/*
 * lsq.h -- C ABI of the GB300 (sm_103a) mixed-precision sketch-and-precondition
 * least-squares solver.
 *
 * Method: Carson & Dauzickaite, "Mixed precision sketching for least-squares
 * problems and its application in GMRES-based iterative refinement",
 * arXiv 2410.06319.  The problem is min_x ||b - A x||_2 with A (m x n) of full
 * rank and m >> n (Sec. 1, Eq. 1.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A is a DEVICE pointer to FP64, row-major, m rows, row stride opts->lda
 *   (elements, >= n; 0 means n).  b is a DEVICE pointer to m FP64 values.
 *   All array arguments are caller-owned device buffers; the library never
 *   frees them and writes only the outputs named in each call.
 * - The handle owns its workspace (device memory, grown on demand) and runs
 *   everything on the CUDA stream given to lsq_create.  Every call below
 *   synchronises that stream once before it returns, so outputs and the info
 *   struct are valid on return.
 * - Arguments are validated before any launch: 1 <= n <= m, n <= s <= m,
 *   tol > 0 and finite, supported precisions, non-null pointers, n <= 1024.
 *   A bad argument returns LSQ_E_INVAL and writes nothing.
 * - Numerical outcomes are statuses, never aborts: iteration caps give
 *   LSQ_NOT_CONVERGED with the last iterate written; device-side waits that
 *   run out give LSQ_E_TIMEOUT; CUDA errors give LSQ_E_CUDA.
 * - The common argument tuple is (A, b, m, n, s, u_s, u_p, u_w, u_r, tol,
 *   seed): u_s = sketch precision (Alg. 1 (sketch)), u_p = QR precision u_QR
 *   (Alg. 1 (QR)), u_w = working precision u (Alg. 2), u_r = residual
 *   precision (Alg. 2 (refinement residual and h = R^-T g)), tol = LSQR and FGMRES tolerance (Sec. 5),
 *   seed = key of the Philox4x32-10 stream that defines the sketch matrix.
 *   A call ignores the members of the tuple it does not use.
 *
 * Sketch matrix.  Omega = s^-1/2 fl_s(G) (Sec. 2 Gaussian embedding, Sec. 5
 * scaling).  G[i, j] (i < s, j < m) is Box-Muller in FP64 of one word pair of
 * Philox4x32-10(counter = (j>>2, i, j>>34, 0), key = (seed lo, seed hi));
 * words 0,1 serve j%4 in {0,1} (cos, sin), words 2,3 serve j%4 in {2,3};
 * U1 = (a+1) 2^-32, U2 = b 2^-32; ln and cos/sin(2 pi U2) are fixed IEEE
 * double sequences (no FMA); fl_s rounds to nearest-even.  G is never stored.
 */
#ifndef LSQ_H
#define LSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Precisions.  F16 = IEEE half (the paper's "half"), BF16 and E4M3 are the
 * GB300 tensor-core formats (sketch only), F32 = single, F64 = double.
 * BF16X3 (sketch only) = single precision on BF16 tensor cores: the sketch
 * operand is fl_bf16(G) and each scaled entry y = fl32(2^k x) of [A | b] is
 * carried by its exact three-term BF16 split hi + lo + lo2, all products
 * accumulated in FP32; its unit roundoff is taken as 2^-24. */
typedef enum lsq_prec {
  LSQ_AUTO = -1,   /* sketch precision only (lsq_lsqr, lsq_lsir and their host/batched forms):
                      the cheapest of BF16, BF16X3, F64 whose sketch gives kappa_est(R) u_s < 1/4
                      (Sec. 3.4: u_s kappa(A) < 1 with kappa(A) estimated from R; kappa_est is the
                      diagonal ratio, a lower bound; a sketch in u_s of an A with kappa(A) > 1/u_s
                      is regularised, its R saturates at a few times 1/u_s and fails the test);
                      info->us_used and info->sketches report the choice */
  LSQ_F64 = 0,
  LSQ_F32 = 1,
  LSQ_F16 = 2,
  LSQ_BF16 = 3,
  LSQ_E4M3 = 4,
  LSQ_BF16X3 = 5,
  LSQ_F64X2 = 6    /* double-double, hi + lo (about 2^-106; stands for the paper's quad, Sec. 5).
                      As u_r: the refinement residual [f; g] = [b - r - A x; -A^T r] of Alg. 2
                      with every product split exactly and summed in double-double, rounded
                      once to FP64.  Not a sketch, QR or working precision. */
} lsq_prec;

typedef enum lsq_status {
  LSQ_OK = 0,
  LSQ_NOT_CONVERGED = 1,   /* iteration cap reached; last iterate written */
  LSQ_E_INVAL = -1,        /* bad argument; nothing written */
  LSQ_E_RANK = -2,         /* R has a zero (or non-finite) diagonal entry */
  LSQ_E_BREAKDOWN = -3,    /* reserved, not returned: a Krylov breakdown ends the method
                              with its current iterate */
  LSQ_E_NONFINITE = -4,    /* a NaN or an infinity in A or b, or a non-finite stage output */
  LSQ_E_CUDA = -5,         /* a CUDA call failed (see lsq_last_cuda_error) */
  LSQ_E_TIMEOUT = -6,      /* a bounded device-side wait ran out */
  LSQ_E_NOMEM = -7,        /* workspace allocation failed */
  LSQ_E_UNSUPPORTED = -8,  /* valid but not supported on this device/build */
  LSQ_E_SIZE = -9          /* larger than the fixed scratch of lsq_qr_r_noalloc */
} lsq_status;

/* info.flags bits */
#define LSQ_WARN_COND 1     /* kappa_est(R) * u_s >= 1: outside Thm 3.1 (Sec. 3.4) */
#define LSQ_INFO_ESCALATED 2 /* refinement re-run with FGMRES products in u^2 (Sec. 5) */

typedef struct lsq_handle lsq_handle;

/* Options.  Zero-initialised fields mean "default" (see lsq_opts_default). */
typedef struct lsq_opts {
  int64_t lda;            /* row stride of A in elements; 0 -> n */
  int32_t lsqr_maxit;     /* LSQR cap; 0 -> 2n (Sec. 5) */
  int32_t ir_maxit;       /* refinement cap; 0 -> 30 (Sec. 5) */
  int32_t gmres_maxit;    /* FGMRES cap per refinement step; 0 -> 50 (Sec. 5) */
  int32_t no_escalate;    /* 1 disables the Sec. 5 re-run of the refinement from (x_0, r_0) with
                             FGMRES products in u^2: u_A = u_L = u_R = double for u = single;
                             double-double (quad) for u = double, with at most
                             max(gmres_maxit, 80) FGMRES iterations (Table 4) */
  int32_t no_colscale;    /* 1 disables the power-of-two column scaling (Sec. 3.2) */
  int32_t ir_stop;        /* refinement stop rule, with dx_i, dr_i the corrections of step i:
                             0: ||dx_i|| <= u||x|| and ||dr_i|| <= u||r||, or (i >= 1) the
                                contraction estimate rho_i = ||dx_i||/||dx_{i-1}|| < 1/2 with
                                rho_i ||dx_i|| <= 4u||x|| (and the same for r), the
                                estimated remaining error at the 4u level of Sec. 5;
                             1: the first test only */
  int32_t timing;         /* 1: time every sketch GEMM and pass launch with CUDA events
                             on the handle's stream (info->kern_ms / kern_launches) */
  int32_t no_graph;       /* 1: launch LSQR / FGMRES iteration batches directly instead of
                             replaying cached CUDA graphs (same arithmetic) */
  int32_t sketch_exact;   /* 1: tensor-core sketch resolves the entries of fl_s(G) whose FP32
                             estimate lies near a rounding midpoint inside the GEMM pipeline;
                             0 (default): the GEMM uses the estimates and a correction kernel
                             adds the exact differences afterwards (same product, faster) */
  double gmres_tol;       /* FGMRES relative-residual tolerance; 0 -> tol */
  double kappa_hint;      /* kappa(A) for the escalation rule; 0 -> estimate from R */
  const double* Y_in;     /* optional device sketch, s x (n+1) column-major (ld = s):
                             skips the sketch inside lsq_qr_r/lsq_lsqr/lsq_lsir */
  const double* R_in;     /* optional device R, n x n column-major upper triangular:
                             skips sketch and QR inside lsq_lsqr/lsq_lsir */
  const double* x0_in;    /* optional device LSQR start (n); used with R_in */
  int64_t sketch_kchunk;  /* tensor-core sketch: at most this many rows of A per split of the
                             m range (each split is summed in FP32, the splits in FP64);
                             0 -> the library's choice */
  int32_t wait_limit_us;  /* limit of each grid-sync wait of the FGMRES Arnoldi step in
                             microseconds; 0 -> 2 s */
  int32_t expire_sync;    /* 1: the Arnoldi step's grid-sync arrival count starts past its
                             completion value, so the first wait runs out after wait_limit_us
                             and the call returns LSQ_E_TIMEOUT (tests the timeout path; the
                             handle stays usable) */
  int32_t sketch_kind;    /* 0: Gaussian embedding (Sec. 2, generated in the GEMM, precision u_s);
                             1: sparse sign embedding (Sec. 2): Omega = zeta^-1/2 (omega_1 ..
                             omega_m), omega_j with sparse_zeta entries +-1 in distinct rows
                             drawn by Floyd's algorithm from Philox4x32-10 (counter (j lo, j hi,
                             call, 1), key = seed); each column of [A | b] rounded to a
                             fixed-point grid 2^-q_c (about 2^-47 of its largest entry) and
                             summed exactly in integers; u_s is then ignored (treated as F64) */
  int32_t sparse_zeta;    /* nonzeros per column of the sparse sign embedding, 1..8; 0 -> 8 */
  int32_t ops_escalated;  /* 1: FGMRES products in u^2 from the first refinement step (FP64 for
                             u_w = F32; double-double for u_w = F64), the products of the Sec. 5
                             re-run */
  double aug_alpha;       /* Sec. 4.1 scaling of the augmented system: FGMRES solves
                             M_L^-1 [[alpha I, A], [A^T, 0]] M_R^-1 [dr/alpha; R dx] =
                             [f; h/alpha], which gives the same correction (dr, dx);
                             0 -> 1 (unscaled, as Sec. 5 runs it); must be finite, >= 0 */
  int32_t h_in_ur;        /* with u_r = LSQ_F64X2: 1 solves h = R^-T g in double-double from the
                             double-double g (Alg. 2 marks this solve with u_r); 0 (default)
                             solves it in FP64 from g rounded to FP64, the reading under which
                             Table 4's escalated rows come out as printed */
  int32_t batch_mode;     /* lsq_lsir_batched: 0 grouped launches when the batch allows them,
                             1 one solve per problem on internal streams */
  int32_t batch_grid;     /* grouped mode: CTAs of the persistent pass launches; 0 -> chosen by
                             timing the candidates on the first call for a batch shape (cached in
                             the handle); every choice gives the same result */
  int32_t arnoldi;        /* FGMRES Arnoldi step (FP64): 0 by vector length (modified Gram-Schmidt
                             from 786,432 rows of [r; x] on, below that classical Gram-Schmidt with a
                             second pass where the first lost more than half of ||w||^2),
                             1 classical with the selective second pass, 2 modified (its work
                             vector in shared memory up to ~4.1e6 rows), 3 modified with the work
                             vector in global memory (the form used past that size) */
} lsq_opts;

/* Diagnostics of one call. */
typedef struct lsq_info {
  int32_t status;
  int32_t flags;
  int32_t lsqr_its;
  int32_t lsqr_flag;        /* 1: ||r|| <= tol||b||, 2: ||Ahat^T r|| test, 3: breakdown, 0: cap */
  int32_t ir_its;
  int32_t gmres_its_total;
  int32_t escalated;
  int32_t ir_converged;
  int32_t gmres_its[32];    /* FGMRES iterations of each refinement step */
  double lsqr_normr;        /* ||b - A x|| estimate at LSQR exit */
  double lsqr_normar;       /* ||Ahat^T r|| estimate at LSQR exit */
  double lsqr_normA;        /* Frobenius-type ||Ahat|| estimate */
  double kappa_R_est;       /* max|r_ii| / min|r_ii| (a lower bound on kappa(R)) */
  double ir_dx_rel;         /* ||dx|| / ||x|| of the last refinement step */
  double ir_dr_rel;         /* ||dr|| / ||r|| of the last refinement step */
  double stage_ms[8];       /* cast, sketch, qr, lsqr, residual, fgmres, update, total */
  int64_t gpu_launches;     /* kernels launched by the call */
  double ir_dx_hist[32];    /* ||dx_i|| / ||x_{i+1}|| of each refinement step */
  double ir_dr_hist[32];    /* ||dr_i|| / ||r_{i+1}|| of each refinement step */
  double gmres_relres[32];  /* FGMRES relative residual reached in each refinement step */
  double kern_ms[8];        /* with opts->timing: summed device time of the sketch GEMM, LSQR
                               pass, FGMRES pass, residual pass, FGMRES Arnoldi step, FGMRES
                               triangular solves and the sketch's deferred correction; one
                               entry spare */
  int64_t kern_launches[8]; /* number of launches behind each kern_ms entry */
  int64_t arnoldi_second_passes; /* FGMRES Arnoldi steps that ran the second Gram-Schmidt pass */
  int32_t us_used;          /* the sketch precision used (the choice of LSQ_AUTO) */
  int32_t sketches;         /* sketches taken (more than one when LSQ_AUTO moved up its ladder) */
  double aug_alpha;         /* the alpha of the augmented system the refinement solved */
} lsq_info;

/* sizeof(lsq_opts) for which = 0, sizeof(lsq_info) for which = 1, else 0: lets
 * bindings check their struct layouts without a GPU. */
size_t lsq_sizeof(int which);

/* Fills *o with the defaults (all zero = defaults). */
void lsq_opts_default(lsq_opts* o);

/* Creates a handle bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Ownership of *h goes to
 * the caller, who releases it with lsq_destroy. */
lsq_status lsq_create(lsq_handle** h, void* cuda_stream);
lsq_status lsq_destroy(lsq_handle* h);

/* Human-readable name of a status; last CUDA error text seen by the handle. */
const char* lsq_status_string(lsq_status st);
const char* lsq_last_cuda_error(const lsq_handle* h);

/*
 * lsq_sketch -- Algorithm 1 (the sketch) (Sec. 3): Y = Omega [A | b] in precision
 * u_s, with the one-sided power-of-two column scaling of Sec. 3.2 (on unless
 * opts->no_colscale) applied before the cast and removed from Y afterwards.
 * F16/BF16 use tcgen05 kind::f16 tensor cores, BF16X3 the same on the three
 * BF16 terms of A, E4M3 kind::f8f6f4, all with FP32 accumulation per split of
 * the m range and an FP64 sum of the splits; F32 and F64 use CUDA cores in
 * that precision.  The FP32 accumulation adds a relative error of about
 * 2^-24 sqrt(k/2) per entry of Y for splits of k rows (k is near m / 5 at the
 * largest m): negligible against the cast for F16/BF16/E4M3, but for BF16X3
 * at m in the millions it, not the cast, sets kappa(A R^-1).  u_w = F32 with
 * u_s = BF16X3 forms the FP32 working copy of A (m x n floats of workspace, as
 * lsq_lsqr does) and the cast reads it where that is exact; any other u_w
 * forms no copy.  Y is the same bit for bit either way.
 * Out: Y, device FP64, s x (n+1) column-major with leading dimension s; its
 * last column is Omega b (used for x_s = R^-1 Q^T Omega b, Sec. 4).
 */
lsq_status lsq_sketch(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                      int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                      double tol, uint64_t seed, const lsq_opts* opts, double* Y);

/*
 * lsq_qr_r -- Algorithm 1 (the QR of the sketch): Householder QR of Y[:, :n] in precision
 * u_p (F32 or F64), reflectors also applied to Y[:, n].  R is normalised to a
 * non-negative diagonal.  Y is computed by lsq_sketch unless opts->Y_in.
 * Out: R, device FP64 n x n column-major (ld = n), upper triangular, values
 * representable in u_p; xs (device, n) = R^-1 (Q^T Omega b), the
 * sketch-and-solve start of Alg. 2 (Sec. 4).  Either output may be NULL.
 */
lsq_status lsq_qr_r(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                    int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                    double tol, uint64_t seed, const lsq_opts* opts, double* R, double* xs);

/*
 * lsq_lsqr -- Algorithm 2 (the LSQR start): LSQR (Paige & Saunders 1982) on A R^-1
 * in working precision u_w (F32 or F64), started from x_s (or opts->x0_in),
 * at most opts->lsqr_maxit (2n) iterations, stopping tests
 * ||r|| <= tol ||b|| or ||Ahat^T r|| <= tol ||Ahat||_est ||r||.
 * Each iteration reads A once (fused A t and A^T q pass) and solves with R
 * and R^T once each.
 * Out: x (device FP64, n).  info may be NULL.
 */
lsq_status lsq_lsqr(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                    int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                    double tol, uint64_t seed, const lsq_opts* opts, double* x, lsq_info* info);

/*
 * lsq_lsir -- Algorithm 2: LSQR start, then augmented-system refinement:
 * [f; g] = [b; 0] - [[I, A], [A^T, 0]] [r; x] in u_r (F64, or double-double
 * for LSQ_F64X2), h = R^-T g in FP64 (or u_r, opts->h_in_ur), split-preconditioned FGMRES (Eq. 1.2,
 * scaled by opts->aug_alpha as in Sec. 4.1; products with Atilde, M_L^-1,
 * M_R^-1 in u_w, Arnoldi and Givens in FP64), update in FP64.  Stops by the rule
 * of opts->ir_stop (by default ||dx|| <= u_w ||x|| and ||dr|| <= u_w ||r||,
 * or the contraction estimate puts the remaining error within 4 u_w), or
 * after opts->ir_maxit steps;
 * then, if not converged and kappa < 1/u_s (kappa_hint, else kappa_est(R)),
 * re-runs the refinement from the LSQR result with the FGMRES products in
 * u_w^2: FP64 for u_w = F32; double-double with at most max(gmres_maxit, 80)
 * FGMRES iterations for u_w = F64 (Sec. 5, Tables 3 and 4).
 * Out: x (device FP64, n) and r = b - A x (device FP64, m; may be NULL).
 */
lsq_status lsq_lsir(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                    int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                    double tol, uint64_t seed, const lsq_opts* opts, double* x, double* r,
                    lsq_info* info);

/*
 * lsq_residual -- the refinement residual of Algorithm 2 (Sec. 4):
 * [f; g] = [b; 0] - [[I, A], [A^T, 0]] [r; x] = [b - r - A x; -A^T r] in u_r:
 * LSQ_F64 (FP64 fused multiply-adds) or LSQ_F64X2 (every product split exactly
 * and summed in double-double, each entry rounded once to FP64).  A (m x n
 * row-major, row stride opts->lda or n), b and r (m) and x (n) are DEVICE FP64
 * arrays, read only; f (m) and g (n) are DEVICE FP64 outputs.  Asynchronous on
 * the handle's stream like the other calls.  LSQ_E_INVAL for a bad argument
 * (nothing written).
 */
lsq_status lsq_residual(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                        lsq_prec u_r, const lsq_opts* opts, const double* x, const double* r,
                        double* f, double* g);

/*
 * lsq_ir_step -- one refinement step of Algorithm 2 from the caller's (x, r):
 * [f; g] = [b - r - A x; -A^T r] in u_r (F64 or LSQ_F64X2), h = R^-T g in FP64
 * (or in u_r with opts->h_in_ur),
 * FGMRES on M_L^-1 Atilde_alpha M_R^-1 [dr/alpha; dz] = [f; h/alpha] (Eq. 1.2 and
 * Sec. 4.1, alpha = opts->aug_alpha or 1; products in u_w, or in u_w^2 with
 * opts->ops_escalated; Arnoldi and
 * Givens in FP64, x0 = 0, at most opts->gmres_maxit iterations, tolerance
 * opts->gmres_tol or tol), then x += R^-1 dz and r += dr.  R is a DEVICE n x n
 * column-major upper-triangular FP64 matrix (e.g. from lsq_qr_r); x (n) and r (m)
 * are DEVICE FP64 vectors, read and overwritten.  info receives the FGMRES
 * iteration count and relative residual (gmres_its[0], gmres_relres[0]) and the
 * relative corrections (ir_dx_rel, ir_dr_rel).  Returns LSQ_OK if FGMRES met its
 * tolerance, LSQ_NOT_CONVERGED if it stopped at its cap (x and r are updated in
 * both cases), or an error status as lsq_lsir (x and r unspecified).
 */
lsq_status lsq_ir_step(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                       int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                       double tol, uint64_t seed, const lsq_opts* opts, const double* R, double* x,
                       double* r, lsq_info* info);

/* One problem of a batch (all pointers are device pointers owned by the caller). */
typedef struct lsq_problem {
  const double* A;   /* m x n row-major FP64, row stride lda (0 -> n) */
  const double* b;   /* m */
  int64_t m, n, s, lda;
  uint64_t seed;     /* key of the problem's sketch matrix */
  double* x;         /* out: n */
  double* r;         /* out: m (may be NULL) */
} lsq_problem;

/*
 * lsq_lsir_host -- lsq_lsir on HOST arrays (the paper has no counterpart: it is
 * the same Algorithm 2 for callers whose data live in host memory).  A (m rows,
 * row stride opts->lda, (m-1)*lda + n elements read) and b (m) are copied into
 * the handle's workspace on its stream (page-locked host memory copies fastest),
 * lsq_lsir runs there, and x (n) and r (m; may be NULL) are copied back to host
 * memory before the call returns.  The workspace keeps a device copy of A until
 * lsq_destroy.  Statuses as lsq_lsir; on an error x and r are not written.
 */
lsq_status lsq_lsir_host(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n,
                         int64_t s, lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r,
                         double tol, uint64_t seed, const lsq_opts* opts, double* x, double* r,
                         lsq_info* info);

/*
 * lsq_lsir_batched -- lsq_lsir on nprob independent problems of uneven sizes
 * (probs is a HOST array of descriptors).
 * Grouped mode (the default when the batch is in its range: u_s in F16, BF16,
 * E4M3, BF16X3; u_p F32 or F64; u_w F32; u_r F64; every n <= 256 and s <= 1024;
 * the Gaussian sketch; no Y_in, R_in, ops_escalated or timing): every stage runs
 * as one grouped launch over all problems -- the cast, one tensor-core sketch
 * grid over every problem's (tile, column group, split) items with per-problem
 * tensor maps and Philox keys, one QR CTA per problem, and one pass launch per
 * LSQR or FGMRES iteration covering every problem's rows, with per-problem done
 * flags -- and the iteration batches replay as CUDA graphs.  A problem's result
 * does not depend on the rest of the batch; it matches lsq_lsir's on the same
 * problem to rounding (the passes and the QR block the work differently).
 * Per-problem mode (opts->batch_mode = 1, or a batch outside that range): the
 * problems run concurrently on up to four internal streams (one worker thread
 * and one workspace per stream, created on first use and owned by the handle),
 * each exactly as lsq_lsir runs it alone.
 * statuses[i] and infos[i] (either may be NULL) receive each problem's outcome;
 * in grouped mode infos[i].stage_ms is not filled.  Returns LSQ_OK if every
 * problem converged, LSQ_NOT_CONVERGED if some did not, or the first error
 * status (a NaN or infinity in any problem's A or b: LSQ_E_NONFINITE for the
 * whole grouped call).
 */
lsq_status lsq_lsir_batched(lsq_handle* h, int32_t nprob, const lsq_problem* probs, lsq_prec u_s,
                            lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol,
                            const lsq_opts* opts, int32_t* statuses, lsq_info* infos);

/*
 * lsq_omega -- the sketch operand fl_s(G)[i, j] for i in [0, s) and
 * j in [j0, j0 + cols), written as FP64 to `out` (device, row-major s x cols),
 * computed by the same device code the sketch kernels use (fast FP32
 * evaluation with the FP64 definition as fallback near rounding boundaries).
 * For testing that the in-kernel Gaussian is the defined one, bit for bit.
 */
lsq_status lsq_omega(lsq_handle* h, int64_t s, int64_t j0, int64_t cols, lsq_prec u_s,
                     uint64_t seed, double* out);

/*
 * lsq_qr_r_noalloc -- the QR of lsq_qr_r (Algorithm 1 (the QR of the sketch)) for callers
 * that cannot allocate.  The paper has no counterpart: this is an interface
 * of this library only.
 *
 * Who needs it: code that may not allocate device memory when it runs, e.g. a
 * service whose device memory is fully committed up front (a fixed budget that
 * must not grow), a latency-critical loop where cudaMalloc / cudaFree would
 * synchronise the device and stall other streams, or a caller that cannot
 * create a handle (lsq_create owns streams and a workspace that grows on
 * demand).  This call allocates nothing, host or device, and needs no handle:
 * its scratch is one file-scope device array of fixed size per device,
 * LSQ_NOALLOC_WORK_BYTES for the working copy of Y plus 64 KiB for the other
 * factors and 256 bytes of control words.
 *
 * In:  Y, device FP64, s x (n+1) column-major with leading dimension s (the
 *      output of lsq_sketch; column n is Omega b).  u_p = LSQ_F32 or LSQ_F64,
 *      the precision of the factorization.  cuda_stream = a cudaStream_t
 *      (NULL = legacy default stream) on which all work is enqueued.
 * Out: R, device FP64 n x n column-major (ld = n), upper triangular with a
 *      non-negative diagonal, the same values lsq_qr_r writes for the same Y
 *      and u_p; c (device FP64, n; may be NULL) = (Q^T Omega b)[:n] with the
 *      same sign normalisation, so that x_s = R^-1 c (Sec. 4).
 *      The caller owns Y, R and c.
 * Limits: 1 <= n <= LSQ_NOALLOC_MAX_N, n <= s <= 16384 (else LSQ_E_INVAL), and
 *      s * (n + 1) * (4 for F32, 8 for F64) <= LSQ_NOALLOC_WORK_BYTES, else
 *      LSQ_E_SIZE before any device work.
 * Errors: LSQ_E_RANK (zero or non-finite diagonal of R), LSQ_E_TIMEOUT (a
 *      bounded grid barrier ran out), LSQ_E_CUDA.  On any error R and c are
 *      unspecified.
 * Synchronisation: returns after the factorization has completed (it
 *      synchronises cuda_stream once to read the scratch's error word).
 * Set-up: the first call on a device, with that device current, looks up the
 *      address of the device's scratch array (cudaGetSymbolAddress); make that
 *      first call before any stream capture begins on the device.  The address
 *      is kept for the life of the process: resetting the device
 *      (cudaDeviceReset) after that first call is not supported.
 * Concurrency: all calls on one device share one scratch array.  Calls that
 *      overlap in time on the same device (from several host threads, or on
 *      several streams) race on it and give wrong results; serialise them.
 *      The scratch's barrier and error words must be zero when the kernels
 *      start: each call clears them on cuda_stream itself.
 */
/*
 * lsq_probe_fma_rate -- measures the device's fused multiply-add throughput
 * (which = 0: FP64, 1: FP32) in FMAs per second on the current device, with
 * independent FMA chains on every SM (best of five timed launches on
 * cuda_stream after one warm-up).  The paper has no counterpart: this is the
 * denominator of the rooflines of the FP64-bound kernels (the residual pass,
 * the Arnoldi step and the FP64 QR), which GB300's narrow FP64 pipe sets.
 * Allocates and frees a few bytes of device memory; synchronises cuda_stream.
 */
lsq_status lsq_probe_fma_rate(int which, void* cuda_stream, double* fma_per_s);

#define LSQ_NOALLOC_WORK_BYTES 8388608
#define LSQ_NOALLOC_MAX_N 1024
lsq_status lsq_qr_r_noalloc(const double* Y, int64_t s, int64_t n, lsq_prec u_p, double* R,
                            double* c, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LSQ_H */
