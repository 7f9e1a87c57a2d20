// Host-side launch wrappers of the device kernels (one stream per call).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace lsq {

// ---------------------------------------------------------------- sketch
// fl_s(G)[i, j0 + c] as FP64 into out (row-major s x cols).
cudaError_t launch_omega(int fmt, int64_t s, int64_t j0, int64_t cols, uint64_t seed, double* out,
                         cudaStream_t st);

// Pass 1 over A: column maxima of [A | b] (as FP64 bit patterns, atomicMax) and,
// when a32 != nullptr, the FP32 working copy (row stride lda32, zero padded).  A NaN
// or an infinity in A or b records DEV_NONFINITE in *err.
cudaError_t launch_colmax_a32(const double* A, int64_t lda, const double* b, int64_t m, int64_t n,
                              unsigned long long* cmax_bits, float* a32, int64_t lda32, int* err,
                              cudaStream_t st);
// Power-of-two exponents k_j (int) from the column maxima (target 2^t, t < 0: none).
cudaError_t launch_scale_exps(const unsigned long long* cmax_bits, int64_t ncols, int t, int* kexp,
                              cudaStream_t st);
// Pass 2 over A: the K-major tensor-core operand Bt: fl_s(2^k_c [A | b][j][c]) for
// column c and data row j, stored in blocks of kBtBlock data rows, each block
// [plane][row c < plane_rows][j % kBtBlock]; rows past n and data rows past m are
// zero.  fmt in {F16, BF16, E4M3, F32, BF16X3}; element size 2, 2, 1, 4, 2;
// BF16X3 has three planes (hi, lo, lo2) of y = fl32(2^k_c x), read from the FP32
// copy a32 (row-major, lda32; may be null) where its power-of-two scaling is exact
// and from A elsewhere.  plane_rows >= n + 1.
constexpr int64_t kBtBlock = 2048;
constexpr int kCast3Rows = 64;   // data rows of a BF16X3 cast tile (32 for the other formats)
int64_t bt_blocks(int64_t m);
size_t bt_bytes(int fmt, int64_t m, int64_t plane_rows);
int64_t cast_row_tiles(int fmt, int64_t m);   // x extent of the cast grid
cudaError_t launch_cast_transpose(int fmt, const double* A, int64_t lda, const double* b, const float* a32,
                                  int64_t lda32, int64_t m, int64_t n, const int* kexp, void* Bt,
                                  int64_t plane_rows, cudaStream_t st);

// Arguments of one tensor-core sketch launch (one problem).
struct SketchTcArgs {
  int64_t s, m, ncols, kchunk, s_pad;
  int bn, nsub, tmem_cols, rows_per_plane;
  int mtiles, ngroups;        // CTA grid of one problem: mtiles x ngroups x splits
  uint32_t k0, k1;
  float* partial;
  int* err;
  // deferred mode: per generator warp a list of the (a, b) pairs whose FP32
  // estimate was too close to a rounding midpoint, packed (data row << 16 | sketch row)
  uint64_t* rec;
  uint32_t* rec_cnt;
  uint32_t rec_cap;
};

// A grouped sketch launch: problem p owns CTAs [start[p], start[p + 1]); tab[p] and
// maps[p] (64-byte aligned, device memory) are its arguments and tensor map.
struct SketchGroup {
  const SketchTcArgs* tab;
  const CUtensorMap* maps;
  const int* start;
  int nprob;
};

// Per-problem arguments of the grouped cast (column maxima and FP32 copy, power-of-two
// column exponents, cast into the blocked Bt layout).
constexpr int64_t kGroupedColmaxRows = 64;
struct GCast {
  const double* A;
  int64_t lda;
  const double* b;
  int64_t m, n;
  unsigned long long* cmax;   // n + 1, zeroed before the launch
  float* a32;                 // FP32 copy (may be null)
  int64_t lda32;
  int* kexp;
  void* Bt;
  int64_t plane_rows;
  int64_t cast_gx;            // row tiles of this problem's cast grid (cast_row_tiles)
};
// Per-problem arguments of the grouped split reduction of the FP32 sketch partials.
struct GReduce {
  const float* partial;
  int splits;
  int64_t ncols, s, s_pad;
  const int* kexp;
  double* Y;
};

struct SketchPlan {
  int fmt;             // FMT_F16, FMT_BF16, FMT_E4M3 (tensor cores) or FMT_F32/F64
  int64_t s, m, ncols; // ncols = n + 1
  int bn;              // columns per CTA (tensor-core path)
  int nsub;            // MMA N-chunks per CTA (1 or 2)
  int ngroups;         // column groups
  int mtiles;          // ceil(s / 128)
  int splits;          // K splits
  int64_t kchunk;      // K extent per split (multiple of the K step)
  int64_t s_pad;       // rows of the partial buffers
  int stages;
  int nt;              // B planes (1, or 3 for the split-term BF16 sketch)
  int rowb;            // bytes per K-major row of a stage (128 or 64)
  size_t smem;
};

// Builds the plan for the tensor-core sketch; returns false if unsupported.
// max_kchunk > 0 caps the rows of A per split (rounded down to whole K steps).
bool plan_sketch_tc(int fmt, int64_t s, int64_t m, int64_t ncols, int num_sms, SketchPlan* p,
                    int64_t max_kchunk = 0);
// Encodes the 3-D TMA descriptor (k within a block, row over all planes, block) of Bt
// (`rows` = planes x plane_rows).
bool encode_bt_tmap(CUtensorMap* tm, const void* Bt, int fmt, int64_t rows, int64_t m, int box_rows,
                    int rowb);
// rec == nullptr: exact mode (FP64 fallbacks resolved inside the kernel).  Otherwise
// deferred mode: the uncertain pairs go to sketch_rec_lists(p) lists of
// sketch_rec_cap(p) entries (counts in rec_cnt) and launch_sketch_fix corrects the
// partials; if it reports *overflow != 0 the exact mode must be rerun.
// The arguments launch_sketch_tc builds for plan p (exact mode), for a grouped table.
SketchTcArgs sketch_tc_args(const SketchPlan& p, uint64_t seed, float* partial, int* err);
// One launch for a batch: ctas = start[nprob]; smem = the largest plan's; every plan must
// have the same format and stage count.
cudaError_t launch_sketch_tc_grouped(int fmt, int stages, const SketchGroup& g, int64_t ctas, size_t smem,
                                     cudaStream_t st);
// Grouped cast: colmax CTAs (ceil(m / kGroupedColmaxRows) per problem), exponent CTAs
// (ceil((n + 1) / 256)), cast CTAs (cast_gx x ceil(plane_rows / 32)); t as in launch_scale_exps.
cudaError_t launch_grouped_cast(int fmt, const GCast* tab, const int* colmax_start, int64_t colmax_ctas,
                                const int* exps_start, int64_t exps_ctas, const int* cast_start,
                                int64_t cast_ctas, int nprob, int t, int* err, cudaStream_t st);
// Grouped sketch_reduce: ceil(s / 256) x (n + 1) CTAs per problem.
cudaError_t launch_grouped_sketch_reduce(const GReduce* tab, const int* start, int64_t ctas, int nprob,
                                         cudaStream_t st);
cudaError_t launch_sketch_tc(const SketchPlan& p, const CUtensorMap& tm, uint64_t seed,
                             float* partial, int* err, cudaStream_t st, uint64_t* rec = nullptr,
                             uint32_t* rec_cnt = nullptr, uint32_t rec_cap = 0);
uint32_t sketch_rec_cap(const SketchPlan& p);
int64_t sketch_rec_lists(const SketchPlan& p);
cudaError_t launch_sketch_fix(const SketchPlan& p, uint64_t seed, const uint64_t* rec,
                              const uint32_t* rec_cnt, uint32_t cap, const double* A, int64_t lda,
                              const double* b, const int* kexp, float* partial, int* overflow,
                              cudaStream_t st);
// CUDA-core sketch in FP64 (fmt F64) or FP32 (fmt F32) from the FP64 data.
cudaError_t launch_sketch_cc(int fmt, const double* A, int64_t lda, const double* b, int64_t m,
                             int64_t n, int64_t s, uint64_t seed, int splits, int64_t kchunk,
                             void* partial, int64_t s_pad, cudaStream_t st);
// Y[c][i] = 2^-k_c s^-1/2 sum_split partial[split][c][i]  (FP64, column-major, ld = s).
cudaError_t launch_sketch_reduce(const void* partial, bool partial_f64, int splits, int64_t ncols,
                                 int64_t s, int64_t s_pad, const int* kexp, double* Y,
                                 cudaStream_t st);

// ---------------------------------------------------------------- sparse sign sketch
// Sec. 2's sparse sign embedding (zeta <= 8 signed rows per data row, exact fixed-point
// sums): Y = Omega [A | b], FP64, column-major with ld = s.  cmax_bits: the column maxima
// of the cast pass.  work: sparse_workspace() bytes.
struct SparsePlan {
  int cb;                 // columns per gather CTA (all n + 1: one CTA per sketch row)
  int colblocks;          // 1
  int splits;             // 1 (each sketch row is summed whole)
  int64_t rows_per_split;
  size_t smem;
};
SparsePlan plan_sparse(int64_t m, int64_t ncols, int s, int num_sms);
size_t sparse_workspace(int64_t m, int64_t ncols, int s, int splits);
cudaError_t launch_sparse_sketch(const SparsePlan& p, const double* A, int64_t lda, const double* b, int64_t m,
                                 int64_t n, int s, int zeta, uint64_t seed,
                                 const unsigned long long* cmax_bits, void* work, double* Y, cudaStream_t st);

// ---------------------------------------------------------------- QR
// Householder QR of Y (s x (n+1), col-major) in FP32 (fp64 = false) or FP64.
// Outputs R (FP64, n x n col-major, diag >= 0) and c (FP64, n).  `work` holds
// s*(n+1) elements of the arithmetic type; `aux` >= (2n + 8) doubles.
cudaError_t launch_qr(bool fp64, const double* Y, int64_t s, int64_t n, void* work, double* aux,
                      unsigned* bar, double* R, double* c, int* err, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------- TRSV
// R (upper) and L = R^T, both column-major n x n with leading dimension ld
// (n rounded up to 16 bytes; padding rows are zero), with the inverses of their
// 32 x 32 diagonal blocks (DU for R, DL for L; 1024 entries per block).
template <typename T>
struct Tri {
  const T* R;
  const T* L;
  const T* DU;
  const T* DL;
  int64_t n;
  int64_t ld;
  int* err = nullptr;   // device error word for bounded waits (may be null)
};
inline int64_t tri_ld(int64_t n, int elem_bytes) {
  const int64_t q = 16 / elem_bytes;
  return (n + q - 1) / q * q;
}

// x = R^-1 y (upper) or x = R^-T y (lower), n <= 1024.  T in {float, double};
// TIN/TOUT any of float/double.  Skips when *done != 0.  With jp, y and x are
// offset on the device by (*jp) * ys and (*jp) * xstr elements.
template <typename T, typename TIN, typename TOUT>
cudaError_t launch_trsv(bool upper, const Tri<T>& f, const TIN* y, double yscale, TOUT* x,
                        const int* done, cudaStream_t st, const int* jp = nullptr, int64_t ys = 0,
                        int64_t xstr = 0);

// Converts R (FP64, col-major) into the FP32 and FP64 factors (R, R^T and the
// diagonal-block inverses); writes max|r_ii| / min|r_ii| to *kappa_est.
cudaError_t launch_prepare_r(const double* R, int64_t n, Tri<float>* f32, Tri<double>* f64,
                             double* kappa_est, cudaStream_t st);

// ---------------------------------------------------------------- passes
int pass_blocks(int num_sms);
// FGMRES pass: az = A z ; Pblk = block sums of v_i A_i (rows of A streamed with
// cp.async.bulk).  With jp, z and v are offset on the device by (*jp) * zs and
// (*jp) * vstr.  Requires A 16-byte aligned with 16-byte rows.
template <typename TA>
cudaError_t launch_pass_fgm(const TA* A, int64_t lda, int64_t m, int64_t n, const TA* z,
                            const TA* v, TA* az, TA* Pblk, int nblk, const int* done, cudaStream_t st,
                            const int* jp, int64_t zs, int64_t vstr, int* err);
// Residual pass (FP64): f_i = b_i - r_i - (A x)_i ; Pblk = block sums of -r_i A_i.
cudaError_t launch_pass_res(const double* A, int64_t lda, int64_t m, int64_t n, const double* x,
                            const double* r, const double* b, double* f, double* Pblk, int nblk,
                            cudaStream_t st);
// out[c] = scale * sum_b P[b][c] (FP64 accumulation).  scale = *scale_ptr * scale_mul
// when scale_ptr != nullptr.
template <typename TP, typename TO>
cudaError_t launch_colsum(const TP* P, int nblk, int64_t n, const double* scale_ptr, double scale_mul,
                          TO* out, const int* done, cudaStream_t st);

}  // namespace lsq
