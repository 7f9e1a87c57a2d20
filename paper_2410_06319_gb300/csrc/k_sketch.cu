// Algorithm 1 (the sketch) (Sec. 3): the sketch Y = Omega [A | b] in precision u_s.
//
//  * cast pass (Sec. 3.2 one-sided scaling): column maxima of [A | b] -> a
//    power-of-two exponent per column -> A_s = fl_s(2^k A) written K-major
//    (one row of Bt per column of A, contiguous over the m data rows), so
//    both tensor-core operands are K-major in 128-byte swizzled tiles.
//  * tcgen05 sketch: per CTA a 128-row slab of the sketch matrix, up to 512
//    columns of [A | b] in TMEM (FP32), a split of the m range.  Warp 0 feeds
//    Bt tiles by TMA, warp 1 issues tcgen05.mma (kind::f16 or kind::f8f6f4),
//    sixteen generator warps synthesise the sketch tile fl_s(G) in registers
//    and store it swizzled into shared memory; four warps drain TMEM into an
//    FP32 partial per split.  G is never stored in global memory.
//  * CUDA-core sketch for u_s = F64 / F32 (no tensor-core format).
//  * reduce: FP64 sum of the split partials, times s^-1/2 and 2^-k_j.
#include <cudaTypedefs.h>

#include <cstring>

#include "cast.cuh"
#include "common.cuh"
#include "gauss.cuh"
#include "kernels.h"

namespace lsq {

// ============================================================ omega test hook
template <int FMT>
__global__ void omega_kernel(int64_t s, int64_t j0, int64_t cols, uint32_t k0, uint32_t k1,
                             double* out) {
  const int64_t q_first = j0 >> 2, q_last = (j0 + cols - 1) >> 2;
  const int64_t nq = q_last - q_first + 1;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= s * nq) return;
  const int64_t i = idx / nq;
  const int64_t q = q_first + idx % nq;
  const uint4 x = philox4x32_10(gauss_counter((uint64_t)q, (uint32_t)i), k0, k1);
  double v[4];
  if constexpr (FMT == FMT_F64 || FMT == FMT_F32) {
    spec_gauss_pair(x.x, x.y, v[0], v[1]);
    spec_gauss_pair(x.z, x.w, v[2], v[3]);
    if constexpr (FMT == FMT_F32) {
#pragma unroll
      for (int t = 0; t < 4; ++t) v[t] = (double)__double2float_rn(v[t]);
    }
  } else {
    uint32_t e0, o0, e1, o1;
    gauss_pair_bits<FMT>(x.x, x.y, e0, o0);
    gauss_pair_bits<FMT>(x.z, x.w, e1, o1);
    v[0] = bits_to_double<FMT>(e0);
    v[1] = bits_to_double<FMT>(o0);
    v[2] = bits_to_double<FMT>(e1);
    v[3] = bits_to_double<FMT>(o1);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int64_t j = q * 4 + t;
    if (j >= j0 && j < j0 + cols) out[i * cols + (j - j0)] = v[t];
  }
}

cudaError_t launch_omega(int fmt, int64_t s, int64_t j0, int64_t cols, uint64_t seed, double* out,
                         cudaStream_t st) {
  const int64_t nq = ((j0 + cols - 1) >> 2) - (j0 >> 2) + 1;
  const int64_t total = s * nq;
  const int threads = 256;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  switch (fmt) {
    case FMT_F64: omega_kernel<FMT_F64><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    case FMT_F32: omega_kernel<FMT_F32><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    case FMT_F16: omega_kernel<FMT_F16><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    case FMT_BF16: omega_kernel<FMT_BF16><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    case FMT_E4M3: omega_kernel<FMT_E4M3><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    case FMT_BF16X3: omega_kernel<FMT_BF16><<<blocks, threads, 0, st>>>(s, j0, cols, k0, k1, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ============================================================ cast pass
// Roundings run on integer units (cast.cuh); the FP64 definition is left only
// for out-of-range values (subnormal results, overflow, subnormal or
// non-finite inputs).

// fl32(2^k x) as FP32 bits, x given by its FP64 bits: integer rounding, else the FP64
// definition (subnormal results, non-finite or subnormal x).
__device__ __forceinline__ uint32_t f32_scaled_bits(uint64_t u, int k) {
  uint32_t b;
  if (f64_scaled_to_f32_bits(u, k, b)) return b;   // normal x, 2^k x in FP32's range
  uint32_t t[3];
  if (cast_terms_int<EncF32>(u, k, t)) return t[0];
  return __float_as_uint(__double2float_rn(ldexp(__longlong_as_double((long long)u), k)));
}

// FP64 bits -> FP32 value, round to nearest even.
__device__ __forceinline__ float f64bits_to_f32(uint64_t u) {
  uint32_t b;
  if (f64_to_f32_bits(u, b)) return __uint_as_float(b);
  return __uint_as_float(f32_scaled_bits(u, 0));
}

__device__ __forceinline__ void colmax_a32_body(const double* __restrict__ A, int64_t lda,
                                                const double* __restrict__ b, int64_t m, int64_t n,
                                                unsigned long long* cmax, float* __restrict__ a32,
                                                int64_t lda32, int64_t rows_per_block, int* err, int64_t blk) {
  const int64_t r0 = blk * rows_per_block;
  const int64_t r1 = min(m, r0 + rows_per_block);
  const int64_t cend = a32 ? max(n + 1, lda32) : n + 1;
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(b);
  constexpr uint64_t kAbs = 0x7FFFFFFFFFFFFFFFull;
  // |v| as FP64 bits is monotone in |v| for non-NaN values: the column maximum
  // is an integer maximum
  for (int64_t c = threadIdx.x; c < cend; c += blockDim.x) {
    uint64_t mx = 0;
    if (c < n) {
      int64_t i = r0;
      for (; i + 8 <= r1; i += 8) {   // eight loads in flight before any use
        uint64_t u[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = __ldcs(Au + (i + q) * lda + c);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          mx = max(mx, u[q] & kAbs);
          if (a32) a32[(i + q) * lda32 + c] = f64bits_to_f32(u[q]);
        }
      }
      for (; i < r1; ++i) {
        const uint64_t u = __ldcs(Au + i * lda + c);
        mx = max(mx, u & kAbs);
        if (a32) a32[i * lda32 + c] = f64bits_to_f32(u);
      }
    } else if (c == n) {
      for (int64_t i = r0; i < r1; ++i) mx = max(mx, bu[i] & kAbs);
      if (a32 && c < lda32)
        for (int64_t i = r0; i < r1; ++i) a32[i * lda32 + c] = 0.0f;
    } else {
      for (int64_t i = r0; i < r1; ++i) a32[i * lda32 + c] = 0.0f;
    }
    if (c <= n && mx > 0) atomicMax(cmax + c, (unsigned long long)mx);
    // |v| bits at or above those of +infinity: an infinity or a NaN in the column
    if (c <= n && mx >= 0x7FF0000000000000ull) set_error(err, DEV_NONFINITE);
  }
}

__global__ void colmax_a32_kernel(const double* __restrict__ A, int64_t lda,
                                  const double* __restrict__ b, int64_t m, int64_t n,
                                  unsigned long long* cmax, float* __restrict__ a32, int64_t lda32,
                                  int64_t rows_per_block, int* err) {
  colmax_a32_body(A, lda, b, m, n, cmax, a32, lda32, rows_per_block, err, blockIdx.x);
}

cudaError_t launch_colmax_a32(const double* A, int64_t lda, const double* b, int64_t m, int64_t n,
                              unsigned long long* cmax_bits, float* a32, int64_t lda32, int* err,
                              cudaStream_t st) {
  const int64_t rows_per_block = 64;
  const unsigned blocks = (unsigned)((m + rows_per_block - 1) / rows_per_block);
  colmax_a32_kernel<<<blocks, 256, 0, st>>>(A, lda, b, m, n, cmax_bits, a32, lda32, rows_per_block, err);
  return cudaGetLastError();
}

__global__ void scale_exps_kernel(const unsigned long long* cmax, int64_t ncols, int t, int* kexp) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const double mx = __longlong_as_double((long long)cmax[c]);
  int k = 0;
  if (t >= 0 && mx > 0.0 && isfinite(mx)) {
    int ex;
    frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1)
    k = t - (ex - 1);
  }
  kexp[c] = k;
}

cudaError_t launch_scale_exps(const unsigned long long* cmax_bits, int64_t ncols, int t, int* kexp,
                              cudaStream_t st) {
  scale_exps_kernel<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(cmax_bits, ncols, t, kexp);
  return cudaGetLastError();
}

template <int FMT>
struct FmtEnc;
template <>
struct FmtEnc<FMT_BF16> {
  using T = EncBF16;
};
template <>
struct FmtEnc<FMT_BF16X3> {
  using T = EncBF16;
};
template <>
struct FmtEnc<FMT_F16> {
  using T = EncF16;
};
template <>
struct FmtEnc<FMT_E4M3> {
  using T = EncE4M3;
};

// The terms of fl_s(2^k x) (x given by its FP64 bits u): integer path, else the
// FP64 definition (round-to-odd into FP32, then to the format).  BF16X3: the three
// BF16 terms of y = fl32(2^k x).
template <int FMT>
__device__ __forceinline__ void cast_bits(uint64_t u, int k, uint32_t (&t)[3]) {
  if constexpr (FMT == FMT_BF16X3) {
    split3_f32(f32_scaled_bits(u, k), t);
  } else if (!cast_terms_int<typename FmtEnc<FMT>::T>(u, k, t)) {
    t[0] = round_f64<FMT>(ldexp(__longlong_as_double((long long)u), k));
  }
}

// Bt layout: blocks of kBtBlock data rows; within a block, [plane][row][k] with
// rows = the padded columns of [A | b] (one row per column) and k contiguous, so a
// sketch CTA's K chunk of its column group lies in one contiguous stretch of a
// few MB (a K-major layout with m-long rows puts every row of a stage on its
// own page once m is in the millions).
template <int FMT>
__device__ __forceinline__ void cast_transpose_body(const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ b, int64_t m, int64_t n,
                                                    const int* __restrict__ kexp, void* __restrict__ Bt,
                                                    int64_t plane_rows, int planes, int64_t bx, int64_t by) {
  __shared__ uint64_t tile[32][33];
  const int64_t j0 = bx * 32, c0 = by * 32;
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(b);
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, c = c0 + threadIdx.x;
    uint64_t v = 0;
    if (j < m) {
      if (c < n) v = __ldcs(Au + j * lda + c);
      else if (c == n) v = bu[j];
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t c = c0 + r, j = j0 + threadIdx.x;
    if (c >= plane_rows) continue;
    // every (row, k) of the padded blocks is written: zeros past column n and row m
    const int64_t blk = j / kBtBlock, kk = j % kBtBlock;
    const int64_t base = (blk * planes * plane_rows + c) * kBtBlock + kk;
    const bool live = c <= n && j < m;
    const uint64_t u = tile[threadIdx.x][r];
    const int k = live ? kexp[c] : 0;
    if constexpr (FMT == FMT_F32) {
      const double v = ldexp(__longlong_as_double((long long)u), k);
      reinterpret_cast<float*>(Bt)[base] = live ? __double2float_rn(v) : 0.0f;
    } else {
      uint32_t tt[3] = {0u, 0u, 0u};
      if (live) cast_bits<FMT>(u, k, tt);
      if constexpr (FMT == FMT_E4M3) {
        reinterpret_cast<uint8_t*>(Bt)[base] = (uint8_t)tt[0];
      } else {
        reinterpret_cast<uint16_t*>(Bt)[base] = (uint16_t)tt[0];
      }
    }
  }
}

// BF16X3: y = fl32(2^k x) in three BF16 planes hi, lo, lo2 (same Bt layout).  Tiles of
// kCast3Rows rows x 32 columns.  y comes from the FP32 copy of A by a power-of-two
// scaling where that is exact (f32_scale_exact), else from the FP64 value (the b
// column, zeros, the bottom of FP32's range, or no FP32 copy); each thread writes two
// consecutive k of a row per plane, so a warp stores 128 contiguous bytes.
__device__ __forceinline__ void cast_bf16x3_body(const double* __restrict__ A, int64_t lda,
                                                 const double* __restrict__ b, const float* __restrict__ a32,
                                                 int64_t lda32, int64_t m, int64_t n,
                                                 const int* __restrict__ kexp, void* __restrict__ Bt,
                                                 int64_t plane_rows, int64_t bx, int64_t by) {
  __shared__ uint32_t tile[32][kCast3Rows + 1];   // [column][row]: y bits
  const int64_t j0 = bx * kCast3Rows, c0 = by * 32;
  const int64_t c = c0 + threadIdx.x;
  const int k = (c <= n) ? kexp[c] : 0;
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(b);
  // the FP32 copy's values of the thread's column, all loads in flight before any use
  constexpr int kPer = kCast3Rows / 8;
  uint32_t av[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int64_t j = j0 + threadIdx.y + 8 * q;
    av[q] = (a32 != nullptr && c < n && j < m) ? __float_as_uint(__ldcs(a32 + j * lda32 + c)) : 0u;
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int r = threadIdx.y + 8 * q;
    const int64_t j = j0 + r;
    uint32_t y = 0;
    if (j < m && c <= n) {
      const bool done = a32 != nullptr && c < n && f32_scale_exact(av[q], k, y);
      if (!done) y = f32_scaled_bits(c < n ? __ldcs(Au + j * lda + c) : bu[j], k);
    }
    tile[threadIdx.x][r] = y;
  }
  __syncthreads();
  uint32_t* P = reinterpret_cast<uint32_t*>(Bt);   // pairs of BF16 values, k even first
  const int64_t pstride = plane_rows * kBtBlock / 2;
  const int64_t j = j0 + 2 * threadIdx.x;
  const int64_t blk = j / kBtBlock, kk = j % kBtBlock;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t cc = c0 + r;
    if (cc >= plane_rows) continue;
    const int64_t base = ((blk * 3 * plane_rows + cc) * kBtBlock + kk) / 2;
    uint32_t t0[3], t1[3];
    split3_f32(tile[r][2 * threadIdx.x], t0);
    split3_f32(tile[r][2 * threadIdx.x + 1], t1);
    P[base] = t0[0] | (t1[0] << 16);
    P[base + pstride] = t0[1] | (t1[1] << 16);
    P[base + 2 * pstride] = t0[2] | (t1[2] << 16);
  }
}

// One-dimensional grid, column tile fastest: the column tiles of a row tile run together,
// so the 128-byte lines that neighbouring tiles share (rows of the FP32 copy need not start
// on a line) are read from DRAM once.
__global__ void cast_bf16x3_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ b,
                                   const float* __restrict__ a32, int64_t lda32, int64_t m, int64_t n,
                                   const int* __restrict__ kexp, void* __restrict__ Bt, int64_t plane_rows) {
  const int64_t ct = (plane_rows + 31) / 32, id = blockIdx.x;
  cast_bf16x3_body(A, lda, b, a32, lda32, m, n, kexp, Bt, plane_rows, id / ct, id % ct);
}

template <int FMT>
__global__ void cast_transpose_kernel(const double* __restrict__ A, int64_t lda,
                                      const double* __restrict__ b, int64_t m, int64_t n,
                                      const int* __restrict__ kexp, void* __restrict__ Bt,
                                      int64_t plane_rows, int planes) {
  cast_transpose_body<FMT>(A, lda, b, m, n, kexp, Bt, plane_rows, planes, blockIdx.x, blockIdx.y);
}

int64_t bt_blocks(int64_t m) { return (m + kBtBlock - 1) / kBtBlock; }

size_t bt_bytes(int fmt, int64_t m, int64_t plane_rows) {
  const int esz = (fmt == FMT_E4M3) ? 1 : (fmt == FMT_F32 ? 4 : 2);
  const int planes = (fmt == FMT_BF16X3) ? 3 : 1;
  return (size_t)bt_blocks(m) * planes * plane_rows * kBtBlock * esz;
}

int64_t cast_row_tiles(int fmt, int64_t m) {
  return bt_blocks(m) * kBtBlock / (fmt == FMT_BF16X3 ? kCast3Rows : 32);
}

cudaError_t launch_cast_transpose(int fmt, const double* A, int64_t lda, const double* b, const float* a32,
                                  int64_t lda32, int64_t m, int64_t n, const int* kexp, void* Bt,
                                  int64_t plane_rows, cudaStream_t st) {
  if (plane_rows < n + 1) return cudaErrorInvalidValue;
  const int planes = (fmt == FMT_BF16X3) ? 3 : 1;
  const int64_t gx = cast_row_tiles(fmt, m);
  if (gx > 2147483647LL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)((plane_rows + 31) / 32));
  dim3 block(32, 8);
  switch (fmt) {
    case FMT_F16: cast_transpose_kernel<FMT_F16><<<grid, block, 0, st>>>(A, lda, b, m, n, kexp, Bt, plane_rows, planes); break;
    case FMT_BF16: cast_transpose_kernel<FMT_BF16><<<grid, block, 0, st>>>(A, lda, b, m, n, kexp, Bt, plane_rows, planes); break;
    case FMT_E4M3: cast_transpose_kernel<FMT_E4M3><<<grid, block, 0, st>>>(A, lda, b, m, n, kexp, Bt, plane_rows, planes); break;
    case FMT_F32: cast_transpose_kernel<FMT_F32><<<grid, block, 0, st>>>(A, lda, b, m, n, kexp, Bt, plane_rows, planes); break;
    case FMT_BF16X3: {
      const int64_t tiles = gx * ((plane_rows + 31) / 32);
      if (tiles > 2147483647LL) return cudaErrorInvalidValue;
      cast_bf16x3_kernel<<<(unsigned)tiles, block, 0, st>>>(A, lda, b, a32, lda32, m, n, kexp, Bt, plane_rows);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ============================================================ tcgen05 sketch
constexpr int kSkGenWarps = 16;
constexpr int kSkGenThreads = kSkGenWarps * 32;
constexpr int kSkFixWarps = 2;                // resolve the FP64 fallbacks of a stage
constexpr int kSkFixThreads = kSkFixWarps * 32;
constexpr int kSkFixFirst = 2 + kSkGenWarps;
constexpr int kSkQMax = 256;                 // FP64 fallbacks queued per stage
// threads of the kernel: TMA + MMA warps, generators, and (exact mode) fixers
__host__ __device__ constexpr int sk_threads(bool defer) {
  return (2 + kSkGenWarps + (defer ? 0 : kSkFixWarps)) * 32;
}

__device__ __forceinline__ void fix_barrier() {
  asm volatile("bar.sync 1, %0;" ::"n"(kSkFixThreads) : "memory");
}

// Smem descriptor for a K-major operand whose rows are ROWB bytes (128: 128-byte
// swizzle; 64: 64-byte swizzle), 8-row core groups 8 * ROWB bytes apart.
template <int ROWB>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)((8u * ROWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;
  return d;
}

// Byte offset of 16-byte chunk kc of row `row` in a swizzled K-major tile.
template <int ROWB>
__device__ __forceinline__ uint32_t swz_chunk(int row, int kc) {
  const int sw = (ROWB == 128) ? (row & 7) : ((row >> 1) & 3);
  return (uint32_t)(row * ROWB + ((kc ^ sw) << 4));
}

// Y partial = fl_s(G)[128 rows] x (sum over NT planes of Bt)[bn columns] over one split of m.
// Exact mode (DEFER = false): pairs whose FP32 estimate is too close to a rounding
// midpoint of u_s are queued per stage and replaced by the FP64 definition by the
// fixer warps before the stage is multiplied.  Deferred mode: the stage is
// multiplied with the FP32 estimates at once and those pairs are recorded;
// sketch_fix_kernel then evaluates them in FP64 and adds (fl_s(G) - estimate) times
// the matching rows of A_s to the partials, which gives the same product.
//
// GROUPED: one launch for a batch of problems.  CTA b belongs to the problem p with
// grp.start[p] <= b < grp.start[p + 1]; its local index gives (tile, column group, split)
// in that problem's grid; the problem's arguments come from grp.tab[p] and its tensor map
// from grp.maps[p] (global memory, written by the host before the launch).
//
// SHARE (deferred mode, two column groups): the CTAs of the two column groups of a
// (tile, split) form a cluster and share the sketch operand: each generates half of the
// 128-row tile (rows 64 r .. 64 r + 63 for cluster rank r) into its own shared memory and
// copies it into its partner's stage with one bulk copy per generator warp, completing the
// partner's full barrier; each MMA commit releases the stage in both CTAs (the empty
// barriers count two arrivals), so neither CTA overwrites a stage its partner still reads.
// Before exiting, the producer waits for the last release of every stage, so no arrival
// from the partner can land in a CTA that has exited.
template <int FMT, int STAGES, int ROWB, int NT, bool DEFER, bool GROUPED, bool SHARE = false>
__global__ void __launch_bounds__(sk_threads(DEFER), 1)
    sketch_tc_kernel(const __grid_constant__ CUtensorMap tmB, const SketchTcArgs a_in, const SketchGroup grp) {
  static_assert(!SHARE || (DEFER && !GROUPED), "operand sharing runs in deferred mode, one problem");
  constexpr int GF = (FMT == FMT_BF16X3) ? FMT_BF16 : FMT;   // format of the sketch operand
  constexpr int EB = (GF == FMT_E4M3) ? 1 : 2;                // bytes per element
  constexpr int BK = ROWB / EB;                               // K elements per stage
  constexpr int EPC = 16 / EB;                                // elements per 16-byte chunk
  constexpr int CPR = ROWB / 16;                              // chunks per row
  constexpr int NCHUNK = 128 * CPR;                           // chunks per sketch tile
  constexpr int PPC = EPC / 2;                                // (a, b) pairs per chunk
  constexpr uint32_t S_BYTES = 128u * ROWB;
  constexpr int KSLICES = ROWB / 32;                          // MMA K slices (32 bytes) per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t mt = blockIdx.x, ng = blockIdx.y, split = blockIdx.z;
  const CUtensorMap* tmp = &tmB;
  int gp = 0;
  if constexpr (GROUPED) {
    gp = group_of(grp.start, grp.nprob, blockIdx.x);
    const int64_t local = (int64_t)blockIdx.x - grp.start[gp];
    const int mtl = grp.tab[gp].mtiles, ngl = grp.tab[gp].ngroups;
    mt = local % mtl;
    ng = (local / mtl) % ngl;
    split = local / ((int64_t)mtl * ngl);
    tmp = grp.maps + gp;
  }
  const SketchTcArgs a = GROUPED ? grp.tab[gp] : a_in;
  const uint32_t b_bytes = (uint32_t)a.bn * ROWB;              // one plane of Bt per stage
  const uint32_t stage_bytes = S_BYTES + NT * b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4 * STAGES + 1);
  uint32_t* qcnt = tslot + 4;                                 // [STAGES]
  uint32_t* qbuf = qcnt + 4;                                  // [STAGES][kSkQMax][3]
  // full: TMA bytes + fixer warps; empty: MMA commit; genned: generator warps done
  // with the FP32 pass; fixed: fallbacks written and the queue reset.
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t genned0 = smem_u32(bars + 2 * STAGES), fixed0 = smem_u32(bars + 3 * STAGES);
  const uint32_t done_bar = smem_u32(bars + 4 * STAGES);

  const int64_t k_begin = split * a.kchunk;
  const int64_t k_end = min(a.m, k_begin + a.kchunk);
  const int nk = (int)((k_end - k_begin + BK - 1) / BK);
  const int chunk = a.bn / a.nsub;
  constexpr uint32_t HALF = S_BYTES / 2;                      // the half tile a CTA generates (SHARE)
  constexpr int GCH = SHARE ? NCHUNK / 2 : NCHUNK;            // chunks this CTA generates per stage
  const uint32_t rank = SHARE ? cl_rank() : 0u;

  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(full0 + 8 * st, DEFER ? 1 + kSkGenWarps : kSkFixWarps + 1);
      mbar_init(empty0 + 8 * st, SHARE ? 2 : 1);
      mbar_init(genned0 + 8 * st, kSkGenWarps);
      mbar_init(fixed0 + 8 * st, kSkFixWarps);
      qcnt[st] = 0;
    }
    mbar_init(done_bar, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tslot), (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tslot;
  if constexpr (SHARE) cl_sync();   // the partner's barriers are initialised before any copy or commit

  if (warp == 0) {
    // ---------------- TMA producer: NT planes x nsub boxes of [chunk rows x ROWB bytes]
    if (lane == 0) {
      if constexpr (GROUPED) {   // the map was written through the generic proxy
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(tmp))
                     : "memory");
      }
      prefetch_tmap(tmp);
      for (int ks = 0; ks < nk; ++ks) {
        const int st = ks % STAGES;
        const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
        if (!mbar_wait(empty0 + 8 * st, ph ^ 1u, a.err, DEV_TIMEOUT_EMPTY)) break;
        mbar_arrive_expect_tx(full0 + 8 * st, (uint32_t)NT * b_bytes + (SHARE ? HALF : 0u));
        const uint32_t sb = smem_u32(smem + st * stage_bytes + S_BYTES);
        const int64_t kx = k_begin + (int64_t)ks * BK;
        const int32_t kin = (int32_t)(kx % kBtBlock), kblk = (int32_t)(kx / kBtBlock);
        for (int t = 0; t < NT; ++t)
          for (int c = 0; c < a.nsub; ++c)
            tma_load_3d(sb + t * b_bytes + (uint32_t)(c * chunk * ROWB), tmp, kin,
                        (int32_t)(t * a.rows_per_plane + ng * a.bn + c * chunk), kblk, full0 + 8 * st);
      }
      if constexpr (SHARE) {
        // tail: the last release of every stage (both MMAs) has arrived here
        for (int st = 0; st < STAGES && st < nk; ++st) {
          const int last = st + ((nk - 1 - st) / STAGES) * STAGES;
          if (!mbar_wait(empty0 + 8 * st, (uint32_t)(last / STAGES) & 1u, a.err, DEV_TIMEOUT_EMPTY)) break;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(GF == FMT_BF16 ? 1u : 0u, 128u, (uint32_t)chunk);
      for (int ks = 0; ks < nk; ++ks) {
        const int st = ks % STAGES;
        const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
        if (!mbar_wait(full0 + 8 * st, ph, a.err, DEV_TIMEOUT_FULL)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * stage_bytes);
        const uint32_t sb = sa + S_BYTES;
#pragma unroll
        for (int kk = 0; kk < KSLICES; ++kk) {
          const uint64_t ad = kmajor_desc<ROWB>(sa + kk * 32);
          for (int c = 0; c < a.nsub; ++c) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
              const uint64_t bd =
                  kmajor_desc<ROWB>(sb + t * b_bytes + (uint32_t)(c * chunk * ROWB) + kk * 32);
              const uint32_t acc = (ks | kk | t) != 0 ? 1u : 0u;
              if constexpr (GF == FMT_E4M3)
                mma_f8(tmem_base + (uint32_t)(c * chunk), ad, bd, idesc, acc);
              else
                mma_f16(tmem_base + (uint32_t)(c * chunk), ad, bd, idesc, acc);
            }
          }
        }
        if constexpr (SHARE) tc_commit_mc(empty0 + 8 * st, (uint16_t)0x3);
        else tc_commit(empty0 + 8 * st);
      }
      tc_commit(done_bar);
    }
  } else if (warp < kSkFixFirst) {
    // ---------------- generator warps: fl_s(G) tile, 128 rows x BK columns
    const int g = threadIdx.x - 64;
    uint32_t wcnt = 0;   // deferred mode: pairs recorded by this warp
    const int64_t cta = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    uint64_t* rec_w = DEFER ? a.rec + (cta * kSkGenWarps + (warp - 2)) * (int64_t)a.rec_cap : nullptr;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % STAGES;
      const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
      if (!mbar_wait(empty0 + 8 * st, ph ^ 1u, a.err, DEV_TIMEOUT_EMPTY)) break;
      if (!DEFER && !mbar_wait(fixed0 + 8 * st, ph ^ 1u, a.err, DEV_TIMEOUT_EMPTY)) break;
      uint8_t* S = smem + st * stage_bytes;
      uint32_t* qb = qbuf + st * (kSkQMax * 3);
      const int64_t kbase = k_begin + (int64_t)ks * BK;
      // SPL threads per 16-byte chunk (two when a half tile has fewer chunks than there are
      // generator threads: each then takes one Philox call and writes 8 bytes)
      constexpr int SPL = (SHARE && EB == 2 && GCH * 2 <= kSkGenThreads) ? 2 : 1;
      constexpr int HPI = (EPC / 4) / SPL;   // Philox calls per thread and chunk
      for (int itm = g; itm < GCH * SPL; itm += kSkGenThreads) {
        const int c = itm / SPL, hp = itm % SPL;
        const int row = c / CPR + (int)rank * 64, kc = c % CPR;
        const uint32_t i = (uint32_t)(mt * 128 + row);
        const uint64_t q0 = (uint64_t)(kbase + kc * EPC) >> 2;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int hh = 0; hh < HPI; ++hh) {
          const int h = hp * HPI + hh;
          const uint4 x = philox4x32_10(gauss_counter(q0 + h, i), a.k0, a.k1);
          uint32_t e0, o0, e1, o1;
          const bool ok0 = gauss_pair_fast<GF>(x.x, x.y, e0, o0);
          const bool ok1 = gauss_pair_fast<GF>(x.z, x.w, e1, o1);
          if constexpr (DEFER) {
            // record the uncertain pairs, in lane order (deterministic lists)
            const unsigned act = __activemask();
            const unsigned m0 = __ballot_sync(act, !ok0), m1 = __ballot_sync(act, !ok1);
            if ((m0 | m1) != 0u) {
              const unsigned lt = (1u << lane) - 1u;
              const uint64_t j0 = (q0 + (uint64_t)h) * 4u;
              if (!ok0) {
                const uint32_t x0 = wcnt + __popc(m0 & lt);
                if (x0 < a.rec_cap) rec_w[x0] = (j0 << 16) | i;
              }
              if (!ok1) {
                const uint32_t x1 = wcnt + __popc(m0) + __popc(m1 & lt);
                if (x1 < a.rec_cap) rec_w[x1] = ((j0 + 2u) << 16) | i;
              }
              wcnt += __popc(m0) + __popc(m1);
            }
          } else if (!ok0 || !ok1) {
#pragma unroll
            for (int p2 = 0; p2 < 2; ++p2) {
              if (p2 == 0 ? ok0 : ok1) continue;
              const uint32_t pa = p2 == 0 ? x.x : x.z, pb = p2 == 0 ? x.y : x.w;
              const uint32_t slot = atomicAdd(qcnt + st, 1u);
              if (slot < (uint32_t)kSkQMax) {
                qb[slot * 3 + 0] = ((uint32_t)row << 8) | ((uint32_t)kc << 4) | (uint32_t)(2 * h + p2);
                qb[slot * 3 + 1] = pa;
                qb[slot * 3 + 2] = pb;
              } else if (p2 == 0) {
                gauss_pair_slow<GF>(pa, pb, e0, o0);   // queue full: resolve in place
              } else {
                gauss_pair_slow<GF>(pa, pb, e1, o1);
              }
            }
          }
          if constexpr (EB == 2) {
            w[2 * hh] = e0 | (o0 << 16);
            w[2 * hh + 1] = e1 | (o1 << 16);
          } else {
            w[hh] = e0 | (o0 << 8) | (e1 << 16) | (o1 << 24);
          }
        }
        if constexpr (SPL == 1)
          *reinterpret_cast<uint4*>(S + swz_chunk<ROWB>(row, kc)) = make_uint4(w[0], w[1], w[2], w[3]);
        else
          *reinterpret_cast<uint2*>(S + swz_chunk<ROWB>(row, kc) + 8 * hp) = make_uint2(w[0], w[1]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if constexpr (SHARE) {
        // this warp's 32 items cover 32 / SPL chunks, whole rows of the tile: one contiguous run
        constexpr int SPLc = (EB == 2 && GCH * 2 <= kSkGenThreads) ? 2 : 1;
        static_assert(GCH * SPLc <= kSkGenThreads && (GCH * SPLc) % 32 == 0 && (32 / SPLc) % CPR == 0,
                      "one item per generator thread, whole rows per warp");
        const int i0 = (warp - 2) * 32;
        if (lane == 0 && i0 < GCH * SPLc) {
          const uint32_t off = (uint32_t)((i0 / SPLc / CPR + (int)rank * 64) * ROWB);
          const uint32_t src = smem_u32(S) + off;
          bulk_s2s(cl_map(src, rank ^ 1u), src, (uint32_t)(32 / SPLc) * 16u, cl_map(full0 + 8 * st, rank ^ 1u));
        }
      }
      if (lane == 0) mbar_arrive(DEFER ? full0 + 8 * st : genned0 + 8 * st);
    }
    if (DEFER && lane == 0) a.rec_cnt[cta * kSkGenWarps + (warp - 2)] = wcnt;
  } else if constexpr (!DEFER) {
    // ---------------- fixer warps: FP64 definition for the queued pairs of a stage,
    // overlapping the generation of the next stage
    const int fx = threadIdx.x - kSkFixFirst * 32;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % STAGES;
      const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
      if (!mbar_wait(genned0 + 8 * st, ph, a.err, DEV_TIMEOUT_FULL)) break;
      uint8_t* S = smem + st * stage_bytes;
      const uint32_t* qb = qbuf + st * (kSkQMax * 3);
      const uint32_t nq = min(qcnt[st], (uint32_t)kSkQMax);
      for (uint32_t qi = fx; qi < nq; qi += kSkFixThreads) {
        const uint32_t pos = qb[qi * 3];
        uint32_t be, bo;
        gauss_pair_slow<GF>(qb[qi * 3 + 1], qb[qi * 3 + 2], be, bo);
        const int row = (int)(pos >> 8), kc = (int)((pos >> 4) & 15), pi = (int)(pos & 15);
        uint8_t* cp = S + swz_chunk<ROWB>(row, kc);
        if constexpr (EB == 2)
          *reinterpret_cast<uint32_t*>(cp + 4 * pi) = be | (bo << 16);
        else
          *reinterpret_cast<uint16_t*>(cp + 2 * pi) = (uint16_t)(be | (bo << 8));
      }
      fence_proxy_async_smem();
      fix_barrier();            // every fixer has read qcnt and written its pairs
      if (fx == 0) qcnt[st] = 0;
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(full0 + 8 * st);
        mbar_arrive(fixed0 + 8 * st);
      }
    }
  }

  // ---------------- epilogue: warps 4..7 drain TMEM lanes 32q .. 32q+31
  if (warp >= 4 && warp < 8) {
    mbar_wait(done_bar, 0, a.err, DEV_TIMEOUT_DONE);
    tc_fence_after();
    const int q = warp & 3;
    const int64_t i = mt * 128 + q * 32 + lane;
    for (int c0 = 0; c0 < a.bn; c0 += 32) {
      uint32_t r[32];
      tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
      tmem_ld_wait();
      if (i < a.s) {
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          const int64_t col = ng * a.bn + c0 + cc;
          if (c0 + cc < a.bn && col < a.ncols)
            a.partial[(split * a.ncols + col) * a.s_pad + i] = __uint_as_float(r[cc]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (SHARE) cl_sync();   // neither CTA leaves while its partner may still copy or commit into it
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, (uint32_t)a.tmem_cols);
  }
}

static int round_up_int(int64_t v, int64_t q) { return (int)(((v + q - 1) / q) * q); }

bool plan_sketch_tc(int fmt, int64_t s, int64_t m, int64_t ncols, int num_sms, SketchPlan* p,
                    int64_t max_kchunk) {
  if (fmt != FMT_F16 && fmt != FMT_BF16 && fmt != FMT_E4M3 && fmt != FMT_BF16X3) return false;
  const int EB = (fmt == FMT_E4M3) ? 1 : 2;
  p->nt = (fmt == FMT_BF16X3) ? 3 : 1;
  p->rowb = (p->nt == 3) ? 64 : 128;
  const int BK = p->rowb / EB;
  p->fmt = fmt;
  p->s = s;
  p->m = m;
  p->ncols = ncols;
  p->ngroups = (int)((ncols + 511) / 512);
  int bn = round_up_int((ncols + p->ngroups - 1) / p->ngroups, 16);
  if (bn > 256) {
    bn = round_up_int(bn, 32);
    p->nsub = 2;
  } else {
    p->nsub = 1;
  }
  p->bn = bn;
  p->mtiles = (int)((s + 127) / 128);
  const size_t stage = (size_t)128 * p->rowb + (size_t)p->nt * bn * p->rowb;
  p->stages = (4 * stage + 1024 + 512 + 4 * kSkQMax * 12 <= 232448) ? 4 : 2;
  p->smem = 1024 + (size_t)p->stages * stage + 512 + (size_t)p->stages * kSkQMax * 12;
  if (p->smem > 232448) return false;
  const int64_t base = (int64_t)p->mtiles * p->ngroups;
  const int64_t ksteps = (m + BK - 1) / BK;
  int64_t splits = (2 * (int64_t)num_sms + base - 1) / base;
  if (splits < 1) splits = 1;
  if (splits > ksteps) splits = ksteps;
  int64_t steps_per = (ksteps + splits - 1) / splits;
  if (max_kchunk == 0 && fmt == FMT_BF16X3) {
    // Single precision on BF16 tensor cores: the FP32 accumulation of one split,
    // not the cast, limits Y once the split is long (the error of the sum grows
    // about linearly with its length, so kappa(A R^-1) does too: 378 at 8e5 rows,
    // 6.8 at 8192 and 3.5 at 2048 for m = 4e6, n = 1000, kappa(A) = 1e7).  Splits of
    // at most kBf16x3Chunk rows, unless their FP32 partials would pass kPartialBudget.
    constexpr int64_t kBf16x3Chunk = 2048;
    constexpr double kPartialBudget = 34359738368.0;   // 32 GiB
    const double per_split = 4.0 * (double)ncols * (double)s;
    const int64_t max_splits = (int64_t)(kPartialBudget / per_split);
    int64_t want = (m + kBf16x3Chunk - 1) / kBf16x3Chunk;
    // at most 25 % more splits, so that the grid fills its last wave of CTAs best
    int64_t best = want, best_idle = -1;
    for (int64_t w = want; w <= want + want / 4; ++w) {
      const int64_t ctas = base * w, waves = (ctas + num_sms - 1) / num_sms;
      const int64_t idle = waves * num_sms - ctas;
      if (best_idle < 0 || idle < best_idle) {
        best = w;
        best_idle = idle;
      }
    }
    want = best;
    if (want > max_splits) want = max_splits;
    if (want > 65535) want = 65535;
    if (want > splits) {
      const int64_t sp = (ksteps + want - 1) / want;
      if (sp < steps_per) steps_per = sp;
    }
  }
  if (max_kchunk > 0) {
    const int64_t cap_steps = max_kchunk / BK > 0 ? max_kchunk / BK : 1;
    if (steps_per > cap_steps) steps_per = cap_steps;
  }
  p->kchunk = steps_per * BK;
  p->splits = (int)((m + p->kchunk - 1) / p->kchunk);
  p->s_pad = s;
  return true;
}

bool encode_bt_tmap(CUtensorMap* tm, const void* Bt, int fmt, int64_t rows, int64_t m, int box_rows,
                    int rowb) {
  // looked up once (thread-safe static initialisation; batched solves call this
  // from several host threads)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  if (!fn) return false;
  const int EB = (fmt == FMT_E4M3) ? 1 : 2;
  if (kBtBlock % (rowb / EB) != 0) return false;   // a stage never straddles two blocks
  // (k within the block, row over all planes, block)
  cuuint64_t dims[3] = {(cuuint64_t)kBtBlock, (cuuint64_t)rows, (cuuint64_t)bt_blocks(m)};
  cuuint64_t strides[2] = {(cuuint64_t)(kBtBlock * EB), (cuuint64_t)(rows * kBtBlock * EB)};
  cuuint32_t box[3] = {(cuuint32_t)(rowb / EB), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(tm, EB == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                  const_cast<void*>(Bt), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int FMT, int STAGES, int ROWB, int NT>
static cudaError_t launch_tc_inst(const SketchPlan& p, const CUtensorMap& tm, const SketchTcArgs& a,
                                  cudaStream_t st) {
  dim3 grid((unsigned)p.mtiles, (unsigned)p.ngroups, (unsigned)p.splits);
  const SketchGroup none{};
  if (a.rec && p.ngroups == 2) {
    // the two column groups of a (tile, split) share the generated operand (a cluster of two)
    auto kern = sketch_tc_kernel<FMT, STAGES, ROWB, NT, true, false, true>;
    cudaError_t e = allow_dyn_smem(kern, (size_t)p.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(sk_threads(true));
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 2;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tm, a, none);
  }
  if (a.rec) {
    auto kern = sketch_tc_kernel<FMT, STAGES, ROWB, NT, true, false>;
    cudaError_t e = allow_dyn_smem(kern, (size_t)p.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, sk_threads(true), p.smem, st>>>(tm, a, none);
  } else {
    auto kern = sketch_tc_kernel<FMT, STAGES, ROWB, NT, false, false>;
    cudaError_t e = allow_dyn_smem(kern, (size_t)p.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, sk_threads(false), p.smem, st>>>(tm, a, none);
  }
  return cudaGetLastError();
}

template <int FMT, int STAGES, int ROWB, int NT>
static cudaError_t launch_tc_grouped_inst(const SketchGroup& g, int64_t ctas, size_t smem, cudaStream_t st) {
  auto kern = sketch_tc_kernel<FMT, STAGES, ROWB, NT, false, true>;
  cudaError_t e = allow_dyn_smem(kern, smem);
  if (e != cudaSuccess) return e;
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  kern<<<(unsigned)ctas, sk_threads(false), smem, st>>>(unused, SketchTcArgs{}, g);
  return cudaGetLastError();
}

cudaError_t launch_sketch_tc(const SketchPlan& p, const CUtensorMap& tm, uint64_t seed,
                             float* partial, int* err, cudaStream_t st, uint64_t* rec,
                             uint32_t* rec_cnt, uint32_t rec_cap) {
  SketchTcArgs a;
  a.s = p.s;
  a.m = p.m;
  a.ncols = p.ncols;
  a.kchunk = p.kchunk;
  a.s_pad = p.s_pad;
  a.bn = p.bn;
  a.nsub = p.nsub;
  a.rows_per_plane = p.ngroups * p.bn;
  a.mtiles = p.mtiles;
  a.ngroups = p.ngroups;
  int tc = 32;
  while (tc < p.bn) tc <<= 1;
  a.tmem_cols = tc;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.partial = partial;
  a.err = err;
  a.rec = rec;
  a.rec_cnt = rec_cnt;
  a.rec_cap = rec_cap;
  const bool four = p.stages == 4;
  switch (p.fmt) {
    case FMT_F16: return four ? launch_tc_inst<FMT_F16, 4, 128, 1>(p, tm, a, st)
                              : launch_tc_inst<FMT_F16, 2, 128, 1>(p, tm, a, st);
    case FMT_BF16: return four ? launch_tc_inst<FMT_BF16, 4, 128, 1>(p, tm, a, st)
                               : launch_tc_inst<FMT_BF16, 2, 128, 1>(p, tm, a, st);
    case FMT_E4M3: return four ? launch_tc_inst<FMT_E4M3, 4, 128, 1>(p, tm, a, st)
                               : launch_tc_inst<FMT_E4M3, 2, 128, 1>(p, tm, a, st);
    case FMT_BF16X3: return four ? launch_tc_inst<FMT_BF16X3, 4, 64, 3>(p, tm, a, st)
                                 : launch_tc_inst<FMT_BF16X3, 2, 64, 3>(p, tm, a, st);
  }
  return cudaErrorInvalidValue;
}

SketchTcArgs sketch_tc_args(const SketchPlan& p, uint64_t seed, float* partial, int* err) {
  SketchTcArgs a{};
  a.s = p.s;
  a.m = p.m;
  a.ncols = p.ncols;
  a.kchunk = p.kchunk;
  a.s_pad = p.s_pad;
  a.bn = p.bn;
  a.nsub = p.nsub;
  a.rows_per_plane = p.ngroups * p.bn;
  a.mtiles = p.mtiles;
  a.ngroups = p.ngroups;
  int tc = 32;
  while (tc < p.bn) tc <<= 1;
  a.tmem_cols = tc;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.partial = partial;
  a.err = err;
  return a;
}

cudaError_t launch_sketch_tc_grouped(int fmt, int stages, const SketchGroup& g, int64_t ctas, size_t smem,
                                     cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 2147483647LL) return cudaErrorInvalidValue;
  const bool four = stages == 4;
  switch (fmt) {
    case FMT_F16: return four ? launch_tc_grouped_inst<FMT_F16, 4, 128, 1>(g, ctas, smem, st)
                              : launch_tc_grouped_inst<FMT_F16, 2, 128, 1>(g, ctas, smem, st);
    case FMT_BF16: return four ? launch_tc_grouped_inst<FMT_BF16, 4, 128, 1>(g, ctas, smem, st)
                               : launch_tc_grouped_inst<FMT_BF16, 2, 128, 1>(g, ctas, smem, st);
    case FMT_E4M3: return four ? launch_tc_grouped_inst<FMT_E4M3, 4, 128, 1>(g, ctas, smem, st)
                               : launch_tc_grouped_inst<FMT_E4M3, 2, 128, 1>(g, ctas, smem, st);
    case FMT_BF16X3: return four ? launch_tc_grouped_inst<FMT_BF16X3, 4, 64, 3>(g, ctas, smem, st)
                                 : launch_tc_grouped_inst<FMT_BF16X3, 2, 64, 3>(g, ctas, smem, st);
  }
  return cudaErrorInvalidValue;
}

// ============================================================ deferred correction
// One block per sketch CTA (same grid): the pairs recorded by its generator warps,
// in list order, 512 at a time.  Phase 1 (one pair per thread, full warps on the
// FP64 pipe): d = fl_s(G) - fl_s(g32) for both entries of the pair; pairs with
// d != 0 are compacted in order.  Phase 2 (one column per thread): for each kept
// pair, partial[i][c] += d * A_s[j][c], with A_s[j][c] recomputed from A by the
// cast's own rounding.  Every partial entry is updated by one thread in a fixed
// order, so the result is deterministic.
constexpr int kFixThreads = 512;

struct SketchFixArgs {
  int64_t s, m, n, ncols, s_pad, lda;
  int bn;
  int share;   // the two column groups shared the operand: read both CTAs' lists
  uint32_t k0, k1, cap;
  const uint64_t* rec;
  const uint32_t* rec_cnt;
  const double* A;
  const double* b;
  const int* kexp;
  float* partial;
  int* overflow;
};

struct FixRec {
  uint32_t i, pad;
  uint64_t j0;
  float de, dodd;   // exact minus estimate: differences of nearby values of the format, exact in FP32
};

template <int FMT>
__global__ void __launch_bounds__(kFixThreads)
    sketch_fix_kernel(const SketchFixArgs f) {
  constexpr int GF = (FMT == FMT_BF16X3) ? FMT_BF16 : FMT;
  __shared__ uint32_t off[2 * kSkGenWarps + 1];
  __shared__ int ovf;
  __shared__ int wsum[kFixThreads / 32];
  __shared__ FixRec kept[kFixThreads];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cta = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
  // with a shared operand, the partner CTA (other column group) generated half of the rows
  const int64_t peer = blockIdx.x + (int64_t)gridDim.x * ((blockIdx.y ^ 1u) + (int64_t)gridDim.y * blockIdx.z);
  const int nl = f.share ? 2 * kSkGenWarps : kSkGenWarps;
  auto list_of = [&](int w) { return (w < kSkGenWarps ? cta : peer) * kSkGenWarps + (w % kSkGenWarps); };
  if (tid == 0) {
    uint32_t o = 0;
    int bad = 0;
    for (int w = 0; w < nl; ++w) {
      const uint32_t c = f.rec_cnt[list_of(w)];
      if (c > f.cap) bad = 1;
      off[w] = o;
      o += min(c, f.cap);
    }
    off[nl] = o;
    ovf = bad;
  }
  __syncthreads();
  if (ovf) {   // lists incomplete: the caller reruns the exact kernel
    if (tid == 0) atomicExch(f.overflow, 1);
    return;
  }
  const uint32_t total = off[nl];
  const int64_t split = blockIdx.z;
  const int64_t col = (int64_t)blockIdx.y * f.bn + tid;
  const bool has_col = tid < f.bn && col < f.ncols;
  const int kc = has_col ? f.kexp[col] : 0;
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(f.A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(f.b);
  for (uint32_t base = 0; base < total; base += kFixThreads) {
    // ---- phase 1: exact minus estimate for one recorded pair
    FixRec r{};
    bool keep = false;
    const uint32_t idx = base + tid;
    if (idx < total) {
      int w = 0;
      while (idx >= off[w + 1]) ++w;
      const uint64_t pk = f.rec[list_of(w) * (int64_t)f.cap + (idx - off[w])];
      r.i = (uint32_t)(pk & 0xFFFFu);
      r.j0 = pk >> 16;
      const uint4 x = philox4x32_10(gauss_counter(r.j0 >> 2, r.i), f.k0, f.k1);
      const uint32_t pa = (r.j0 & 2u) ? x.z : x.x, pb = (r.j0 & 2u) ? x.w : x.y;
      uint32_t fe, fo, xe, xo;
      gauss_pair_fast<GF>(pa, pb, fe, fo);
      gauss_pair_slow<GF>(pa, pb, xe, xo);
      r.de = __fsub_rn(bits_to_float<GF>(xe), bits_to_float<GF>(fe));
      r.dodd = __fsub_rn(bits_to_float<GF>(xo), bits_to_float<GF>(fo));
      keep = (r.de != 0.0f || r.dodd != 0.0f) && (int64_t)r.i < f.s;
    }
    // ---- ordered compaction of the kept pairs
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, nkept = 0;
    for (int q = 0; q < kFixThreads / 32; ++q) {
      if (q < warp) before += wsum[q];
      nkept += wsum[q];
    }
    if (keep) kept[before + __popc(bal & ((1u << lane) - 1u))] = r;
    __syncthreads();
    // ---- phase 2: partial[i][col] += d * A_s[j][col], in FP32 like the GEMM.  d is one
    // step of the format (a power of two) or the difference of two nearby values of it,
    // and A_s[j][col] has at most 24 significant bits (BF16X3: hi + lo + lo2, exact in
    // FP32), so each product is exact; the two of a pair are summed in FP32.
    if (has_col) {
      float* pc = f.partial + (split * f.ncols + col) * f.s_pad;
      for (int q = 0; q < nkept; ++q) {
        const FixRec& k = kept[q];
        float add = 0.0f;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float d = e ? k.dodd : k.de;
          const int64_t j = (int64_t)k.j0 + e;
          if (d == 0.0f || j >= f.m) continue;
          const uint64_t u = (col < f.n) ? Au[j * f.lda + col] : bu[j];
          uint32_t t[3];
          cast_bits<FMT>(u, kc, t);
          float v = bits_to_float<GF>(t[0]);
          if constexpr (FMT == FMT_BF16X3)
            v = __fadd_rn(__fadd_rn(v, bits_to_float<GF>(t[1])), bits_to_float<GF>(t[2]));
          add = __fmaf_rn(d, v, add);
        }
        pc[k.i] += add;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_sketch_fix(const SketchPlan& p, uint64_t seed, const uint64_t* rec,
                              const uint32_t* rec_cnt, uint32_t cap, const double* A, int64_t lda,
                              const double* b, const int* kexp, float* partial, int* overflow,
                              cudaStream_t st) {
  if (p.bn > kFixThreads) return cudaErrorInvalidValue;
  SketchFixArgs f;
  f.s = p.s;
  f.m = p.m;
  f.n = p.ncols - 1;
  f.ncols = p.ncols;
  f.s_pad = p.s_pad;
  f.lda = lda;
  f.bn = p.bn;
  f.share = p.ngroups == 2 ? 1 : 0;   // launch_sketch_tc shares the operand exactly then (deferred mode)
  f.k0 = (uint32_t)seed;
  f.k1 = (uint32_t)(seed >> 32);
  f.cap = cap;
  f.rec = rec;
  f.rec_cnt = rec_cnt;
  f.A = A;
  f.b = b;
  f.kexp = kexp;
  f.partial = partial;
  f.overflow = overflow;
  dim3 grid((unsigned)p.mtiles, (unsigned)p.ngroups, (unsigned)p.splits);
  switch (p.fmt) {
    case FMT_F16: sketch_fix_kernel<FMT_F16><<<grid, kFixThreads, 0, st>>>(f); break;
    case FMT_BF16: sketch_fix_kernel<FMT_BF16><<<grid, kFixThreads, 0, st>>>(f); break;
    case FMT_E4M3: sketch_fix_kernel<FMT_E4M3><<<grid, kFixThreads, 0, st>>>(f); break;
    case FMT_BF16X3: sketch_fix_kernel<FMT_BF16X3><<<grid, kFixThreads, 0, st>>>(f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Records per generator warp for deferred correction: the warp sees 4 * kchunk
// (a, b) pairs; expected fractions near a midpoint are ~0.2% (BF16), ~1.6%
// (FP16), ~0.01% (E4M3), so the capacity leaves a 4x or larger margin.
uint32_t sketch_rec_cap(const SketchPlan& p) {
  const int64_t pairs = 4 * p.kchunk;
  const int64_t div = (p.fmt == FMT_F16) ? 16 : (p.fmt == FMT_E4M3) ? 1024 : 128;
  return (uint32_t)(pairs / div + 64);
}
int64_t sketch_rec_lists(const SketchPlan& p) {
  return (int64_t)p.mtiles * p.ngroups * p.splits * kSkGenWarps;
}

// ============================================================ CUDA-core sketch
// CTA tile: 16 sketch rows x 256 columns of [A | b]; K step 16; 256 threads,
// each 4 rows x 4 columns.  The sketch tile is generated once per K step.
template <typename T>
__global__ void __launch_bounds__(256)
    sketch_cc_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ b,
                     int64_t m, int64_t n, int64_t s, uint32_t k0, uint32_t k1, int64_t kchunk,
                     T* __restrict__ partial, int64_t s_pad) {
  constexpr int BM = 16, BN = 256, BKc = 16;
  __shared__ T Gs[BKc][BM];
  __shared__ T Bs[BKc][BN];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * BM, c0 = (int64_t)blockIdx.y * BN;
  const int64_t split = blockIdx.z;
  const int64_t kb = split * kchunk, ke = min(m, kb + kchunk);
  const int tr = (tid >> 6) * 4, tc = (tid & 63) * 4;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
  for (int64_t k = kb; k < ke; k += BKc) {
    // sketch tile: 16 rows x 16 K -> 64 Philox calls (4 K each)
    if (tid < 64) {
      const int r = tid >> 2, qq = tid & 3;
      const int64_t j = k + qq * 4;
      const uint4 x = philox4x32_10(gauss_counter((uint64_t)j >> 2, (uint32_t)(i0 + r)), k0, k1);
      double v[4];
      spec_gauss_pair(x.x, x.y, v[0], v[1]);
      spec_gauss_pair(x.z, x.w, v[2], v[3]);
#pragma unroll
      for (int t = 0; t < 4; ++t) Gs[qq * 4 + t][r] = (T)v[t];  // T = float rounds to nearest
    }
    for (int e = tid; e < BKc * BN; e += 256) {
      const int kk = e / BN, cc = e % BN;
      const int64_t j = k + kk, c = c0 + cc;
      double v = 0.0;
      if (j < ke) {
        if (c < n) v = A[j * lda + c];
        else if (c == n) v = b[j];
      }
      Bs[kk][cc] = (T)v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKc; ++kk) {
      T gv[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) gv[x] = Gs[kk][tr + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) bv[y] = Bs[kk][tc + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(gv[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int64_t c = c0 + tc + y;
    if (c > n) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t i = i0 + tr + x;
      if (i < s) partial[(split * (n + 1) + c) * s_pad + i] = acc[x][y];
    }
  }
}

cudaError_t launch_sketch_cc(int fmt, const double* A, int64_t lda, const double* b, int64_t m,
                             int64_t n, int64_t s, uint64_t seed, int splits, int64_t kchunk,
                             void* partial, int64_t s_pad, cudaStream_t st) {
  dim3 grid((unsigned)((s + 15) / 16), (unsigned)((n + 1 + 255) / 256), (unsigned)splits);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (fmt == FMT_F64)
    sketch_cc_kernel<double><<<grid, 256, 0, st>>>(A, lda, b, m, n, s, k0, k1, kchunk,
                                                   static_cast<double*>(partial), s_pad);
  else if (fmt == FMT_F32)
    sketch_cc_kernel<float><<<grid, 256, 0, st>>>(A, lda, b, m, n, s, k0, k1, kchunk,
                                                  static_cast<float*>(partial), s_pad);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ============================================================ split reduce
// FP64 partials: an FP64 sum.  FP32 partials (the tensor-core splits): Knuth's TwoSum
// in FP32, an error-free transformation of each addition, with the rounding errors
// collected in a second FP32 word; hi + lo carries the sum of the splits to about
// 2^-48 relative (double-float), on the FP32 pipe instead of GB300's narrow FP64 pipe
// (the sum over thousands of 2048-row splits at m = 4e6 is 8e9 additions).
template <typename TP>
__device__ __forceinline__ void sketch_reduce_body(const TP* __restrict__ partial, int splits, int64_t ncols,
                                                   int64_t s, int64_t s_pad, const int* __restrict__ kexp,
                                                   double inv_sqrt_s, double* __restrict__ Y, int64_t bx,
                                                   int64_t c) {
  const int64_t i = bx * (int64_t)blockDim.x + threadIdx.x;
  if (i >= s) return;
  double acc;
  if constexpr (sizeof(TP) == 8) {
    acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) acc += (double)partial[((int64_t)sp * ncols + c) * s_pad + i];
  } else {
    float hi = 0.0f, lo = 0.0f;
    const TP* p = partial + c * s_pad + i;
    const int64_t stride = ncols * s_pad;
    for (int sp = 0; sp < splits; ++sp) {
      const float x = __ldcs(p + (int64_t)sp * stride);
      const float t = __fadd_rn(hi, x);
      const float xb = __fsub_rn(t, hi);
      const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, xb)), __fsub_rn(x, xb));
      hi = t;
      lo = __fadd_rn(lo, err);
    }
    acc = (double)hi + (double)lo;
  }
  const int k = kexp ? kexp[c] : 0;
  Y[c * s + i] = ldexp(acc * inv_sqrt_s, -k);
}

template <typename TP>
__global__ void sketch_reduce_kernel(const TP* __restrict__ partial, int splits, int64_t ncols,
                                     int64_t s, int64_t s_pad, const int* __restrict__ kexp,
                                     double inv_sqrt_s, double* __restrict__ Y) {
  sketch_reduce_body<TP>(partial, splits, ncols, s, s_pad, kexp, inv_sqrt_s, Y, blockIdx.x, blockIdx.y);
}

// ============================================================ grouped (batched) forms
// One launch per stage for a batch of problems: CTA b works for the problem p with
// start[p] <= b < start[p + 1] (start: prefix sums of the per-problem CTA counts), on
// the block of that problem's own grid given by b - start[p].  Per-problem arguments
// come from a device table.
__global__ void grouped_colmax_kernel(const GCast* __restrict__ tab, const int* __restrict__ start, int nprob,
                                      int* err) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GCast& g = tab[p];
  colmax_a32_body(g.A, g.lda, g.b, g.m, g.n, g.cmax, g.a32, g.lda32, kGroupedColmaxRows, err,
                  (int64_t)blockIdx.x - start[p]);
}

__global__ void grouped_scale_exps_kernel(const GCast* __restrict__ tab, const int* __restrict__ start,
                                          int nprob, int t) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GCast& g = tab[p];
  const int64_t c = ((int64_t)blockIdx.x - start[p]) * blockDim.x + threadIdx.x;
  if (c > g.n) return;
  const double mx = __longlong_as_double((long long)g.cmax[c]);
  int k = 0;
  if (t >= 0 && mx > 0.0 && isfinite(mx)) {
    int ex;
    frexp(mx, &ex);
    k = t - (ex - 1);
  }
  g.kexp[c] = k;
}

template <int FMT>
__global__ void grouped_cast_kernel(const GCast* __restrict__ tab, const int* __restrict__ start, int nprob,
                                    int planes) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GCast& g = tab[p];
  const int64_t local = (int64_t)blockIdx.x - start[p];
  if constexpr (FMT == FMT_BF16X3) {   // column tile fastest, as cast_bf16x3_kernel
    const int64_t ct = (g.plane_rows + 31) / 32;
    cast_bf16x3_body(g.A, g.lda, g.b, g.a32, g.lda32, g.m, g.n, g.kexp, g.Bt, g.plane_rows, local / ct, local % ct);
  } else {
    cast_transpose_body<FMT>(g.A, g.lda, g.b, g.m, g.n, g.kexp, g.Bt, g.plane_rows, planes, local % g.cast_gx,
                             local / g.cast_gx);
  }
}

__global__ void grouped_sketch_reduce_kernel(const GReduce* __restrict__ tab, const int* __restrict__ start,
                                             int nprob) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GReduce& g = tab[p];
  const int64_t local = (int64_t)blockIdx.x - start[p];
  const int64_t gx = (g.s + 255) / 256;
  sketch_reduce_body<float>(g.partial, g.splits, g.ncols, g.s, g.s_pad, g.kexp, 1.0 / sqrt((double)g.s), g.Y,
                            local % gx, local / gx);
}

cudaError_t launch_grouped_cast(int fmt, const GCast* tab, const int* colmax_start, int64_t colmax_ctas,
                                const int* exps_start, int64_t exps_ctas, const int* cast_start,
                                int64_t cast_ctas, int nprob, int t, int* err, cudaStream_t st) {
  if (colmax_ctas > 2147483647LL || cast_ctas > 2147483647LL) return cudaErrorInvalidValue;
  grouped_colmax_kernel<<<(unsigned)colmax_ctas, 256, 0, st>>>(tab, colmax_start, nprob, err);
  grouped_scale_exps_kernel<<<(unsigned)exps_ctas, 256, 0, st>>>(tab, exps_start, nprob, t);
  const int planes = (fmt == FMT_BF16X3) ? 3 : 1;
  const dim3 block(32, 8);
  switch (fmt) {
    case FMT_F16: grouped_cast_kernel<FMT_F16><<<(unsigned)cast_ctas, block, 0, st>>>(tab, cast_start, nprob, planes); break;
    case FMT_BF16: grouped_cast_kernel<FMT_BF16><<<(unsigned)cast_ctas, block, 0, st>>>(tab, cast_start, nprob, planes); break;
    case FMT_E4M3: grouped_cast_kernel<FMT_E4M3><<<(unsigned)cast_ctas, block, 0, st>>>(tab, cast_start, nprob, planes); break;
    case FMT_BF16X3: grouped_cast_kernel<FMT_BF16X3><<<(unsigned)cast_ctas, block, 0, st>>>(tab, cast_start, nprob, planes); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_grouped_sketch_reduce(const GReduce* tab, const int* start, int64_t ctas, int nprob,
                                         cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  grouped_sketch_reduce_kernel<<<(unsigned)ctas, 256, 0, st>>>(tab, start, nprob);
  return cudaGetLastError();
}

cudaError_t launch_sketch_reduce(const void* partial, bool partial_f64, int splits, int64_t ncols,
                                 int64_t s, int64_t s_pad, const int* kexp, double* Y,
                                 cudaStream_t st) {
  dim3 grid((unsigned)((s + 255) / 256), (unsigned)ncols);
  const double inv = 1.0 / sqrt((double)s);
  if (partial_f64)
    sketch_reduce_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(partial), splits,
                                                       ncols, s, s_pad, kexp, inv, Y);
  else
    sketch_reduce_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(partial), splits,
                                                      ncols, s, s_pad, kexp, inv, Y);
  return cudaGetLastError();
}

}  // namespace lsq
