// The sparse sign embedding of Sec. 2 as the sketch of Algorithm 1: Omega =
// zeta^-1/2 (omega_1 ... omega_m), omega_j with zeta entries +-1 in distinct rows.
//
//  * rows kernel: for each data row j, Philox4x32-10 (counter (j lo, j hi, call, 1),
//    key (seed lo, seed hi)) gives eight words; Floyd's algorithm draws the zeta rows
//    without replacement (k = 0..zeta-1, t = s - zeta + k, r = (w_k (t + 1)) >> 32,
//    row r unless already chosen, else row t), the sign of the k-th row is - if w_k is
//    odd; entries of a table (row | sign << 15) and a count of data rows per sketch row.
//  * grid kernel: per column c of [A | b] the exponent q_c of a fixed-point grid 2^-q_c
//    with max|a_c| 2^q_c <= 2^(61 - h), h the bit length of the largest count, so no
//    sum of a sketch row's entries leaves 62 bits.
//  * sketch kernel: each CTA owns a block of CB columns (and a slice of the data rows)
//    and adds the rounded entries (round half even on the grid, integer arithmetic on
//    the FP64 bits) into int64 accumulators in shared memory with integer atomics: exact,
//    so the result does not depend on the order.  A warp takes one data row per step,
//    lane = (k, c): the zeta rows of a data row are distinct, so its lanes never collide.
//  * finalize: the exact sum of the row slices, converted once to FP64, times 2^-q_c and
//    zeta^-1/2 (the same operations in the same order as the definition, so Y is exact).
// HBM: [A | b] is read once; the row table (16 bytes per data row) is re-read per column
// block and stays in L2.
#include <cstdint>

#include "common.cuh"
#include "gauss.cuh"
#include "kernels.h"

namespace lsq {

constexpr int kSpMaxZeta = 8;

__global__ void sparse_rows_kernel(int64_t m, int s, int zeta, uint32_t k0, uint32_t k1,
                                   uint16_t* __restrict__ table, unsigned* __restrict__ counts) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m) return;
  uint32_t w[8];
#pragma unroll
  for (int call = 0; call < 2; ++call) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)call, 1u),
                                  k0, k1);
    w[4 * call + 0] = x.x;
    w[4 * call + 1] = x.y;
    w[4 * call + 2] = x.z;
    w[4 * call + 3] = x.w;
  }
  int rows[kSpMaxZeta];
#pragma unroll
  for (int k = 0; k < kSpMaxZeta; ++k) {
    if (k >= zeta) break;
    const uint32_t t = (uint32_t)(s - zeta + k);
    const uint32_t r = (uint32_t)(((uint64_t)w[k] * (uint64_t)(t + 1u)) >> 32);
    bool taken = false;
#pragma unroll
    for (int q = 0; q < kSpMaxZeta; ++q)
      if (q < k && rows[q] == (int)r) taken = true;
    rows[k] = taken ? (int)t : (int)r;
    table[j * kSpMaxZeta + k] = (uint16_t)(rows[k] | ((w[k] & 1u) << 15));
    atomicAdd(counts + rows[k], 1u);
  }
}

// q_c = (61 - h) - e_c, e_c the binary exponent of max|a_c| (max = f 2^e, f in [0.5, 1));
// 0 for an all-zero column.  One block: first the largest count.
__global__ void sparse_grid_kernel(const unsigned long long* __restrict__ cmax_bits, int64_t ncols,
                                   const unsigned* __restrict__ counts, int s, int* __restrict__ qexp) {
  __shared__ unsigned red[32];
  unsigned mx = 0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) mx = max(mx, counts[i]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const int h = 32 - __clz((int)red[0]);   // bit length of the largest count
  for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
    const uint64_t u = cmax_bits[c];       // |max| as FP64 bits (finite: the cast pass checked)
    int q = 0;
    if (u != 0) {
      const int E = (int)(u >> 52);
      int e;
      if (E > 0) {
        e = E - 1022;                      // f in [0.5, 1): 2^(E-1023) (1.x) = 0.1x 2^(E-1022)
      } else {                             // subnormal: leading bit position of the fraction
        const uint64_t f = u & 0xFFFFFFFFFFFFFull;
        e = (63 - __clzll((long long)f)) - 1074 + 1;
      }
      q = (61 - h) - e;
    }
    qexp[c] = q;
  }
}

// round(x 2^q) to the nearest integer, ties to even, from the FP64 bits of x (the grid
// exponents keep |result| <= 2^61).
__device__ __forceinline__ long long to_grid(uint64_t u, int q) {
  const int E = (int)((u >> 52) & 0x7FF);
  long long M = (long long)(u & 0xFFFFFFFFFFFFFull);
  if (E > 0) M |= (1ll << 52);
  if (M == 0) return 0;
  const int sh = (E > 0 ? E : 1) - 1075 + q;
  long long v;
  if (sh >= 0) {
    v = M << sh;
  } else if (sh <= -64) {
    v = 0;
  } else {
    const int r = -sh;
    long long qv = (r >= 63) ? 0 : (M >> r);
    const long long rem = (r >= 63) ? M : (M - (qv << r));
    const long long half = 1ll << (r - 1);
    if (rem > half || (rem == half && (qv & 1))) qv += 1;
    v = qv;
  }
  return (u >> 63) ? -v : v;
}

constexpr int kSpThreads = 512;

template <int CB>
__global__ void __launch_bounds__(kSpThreads)
    sparse_sketch_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ b, int64_t m,
                         int64_t n, int s, int zeta, const uint16_t* __restrict__ table,
                         const int* __restrict__ qexp, long long* __restrict__ part, int64_t rows_per_split) {
  extern __shared__ __align__(16) long long acc[];   // [s][CB]
  const int64_t c0 = (int64_t)blockIdx.x * CB;
  const int64_t split = blockIdx.y;
  const int64_t ncols = n + 1;
  for (int i = threadIdx.x; i < s * CB; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int KPW = 32 / CB;                  // table entries a lane group covers per step
  const int k = lane / CB, cc = lane % CB;      // lane -> (target slot, column)
  const int64_t c = c0 + cc;
  const bool col_ok = c < ncols;
  const int q = col_ok ? qexp[c] : 0;
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(b);
  const int64_t r0 = split * rows_per_split, r1 = min(m, r0 + rows_per_split);
  for (int64_t j = r0 + warp; j < r1; j += nw) {
    const uint64_t u = col_ok ? (c < n ? __ldcs(Au + j * lda + c) : __ldcs(bu + j)) : 0ull;
    const long long v = to_grid(u, q);
    // 32 / CB >= 8 lane groups: every slot of the row in one step
    for (int kk = k; kk < zeta; kk += KPW) {
      if (!col_ok) break;
      const uint16_t t = table[j * kSpMaxZeta + kk];
      const int row = t & 0x7FFF;
      const long long sv = (t >> 15) ? -v : v;
      atomicAdd(reinterpret_cast<unsigned long long*>(acc + row * CB + cc), (unsigned long long)sv);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s * CB; i += blockDim.x) {
    const int cl = i / s, row = i % s;
    const int64_t col = c0 + cl;
    if (col < ncols) part[(split * ncols + col) * s + row] = acc[row * CB + cl];
  }
}

__global__ void sparse_finalize_kernel(const long long* __restrict__ part, int splits, int64_t ncols, int s,
                                       const int* __restrict__ qexp, double scale, double* __restrict__ Y) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncols * s) return;
  const int64_t c = idx / s;
  long long t = 0;
  for (int sp = 0; sp < splits; ++sp) t += part[(int64_t)sp * ncols * s + idx];
  Y[idx] = ldexp((double)t, -qexp[c]) * scale;
}

size_t sparse_workspace(int64_t m, int64_t ncols, int s, int splits) {
  return (size_t)m * kSpMaxZeta * 2 + (size_t)s * 4 + (size_t)ncols * 4 +
         (size_t)splits * (size_t)ncols * (size_t)s * 8 + 1024;
}

SparsePlan plan_sparse(int64_t m, int64_t ncols, int s, int num_sms) {
  SparsePlan p{};
  p.cb = (int64_t)s * 4 * 8 <= 200 * 1024 ? 4 : ((int64_t)s * 2 * 8 <= 200 * 1024 ? 2 : 1);
  p.colblocks = (int)((ncols + p.cb - 1) / p.cb);
  const int per_sm = (int)((227 * 1024) / ((size_t)s * p.cb * 8));
  const int64_t want = 2ll * num_sms * (per_sm > 0 ? per_sm : 1);
  int64_t splits = (want + p.colblocks - 1) / p.colblocks;
  const int64_t max_by_rows = (m + 4095) / 4096;          // at least 4096 data rows a split
  if (splits > max_by_rows) splits = max_by_rows;
  const double budget = 2147483648.0;                      // int64 partials, at most 2 GiB
  const int64_t max_by_mem = (int64_t)(budget / (8.0 * (double)ncols * s));
  if (splits > max_by_mem) splits = max_by_mem;
  if (splits < 1) splits = 1;
  p.rows_per_split = (m + splits - 1) / splits;
  p.splits = (int)((m + p.rows_per_split - 1) / p.rows_per_split);
  p.smem = (size_t)s * p.cb * 8;
  return p;
}

cudaError_t launch_sparse_sketch(const SparsePlan& p, const double* A, int64_t lda, const double* b, int64_t m,
                                 int64_t n, int s, int zeta, uint64_t seed,
                                 const unsigned long long* cmax_bits, void* work, double* Y, cudaStream_t st) {
  if (zeta < 1 || zeta > kSpMaxZeta || zeta > s || s > 16384) return cudaErrorInvalidValue;
  const int64_t ncols = n + 1;
  auto* base = static_cast<unsigned char*>(work);
  auto* table = reinterpret_cast<uint16_t*>(base);
  size_t off = ((size_t)m * kSpMaxZeta * 2 + 255) & ~(size_t)255;
  auto* counts = reinterpret_cast<unsigned*>(base + off);
  off = (off + (size_t)s * 4 + 255) & ~(size_t)255;
  auto* qexp = reinterpret_cast<int*>(base + off);
  off = (off + (size_t)ncols * 4 + 255) & ~(size_t)255;
  auto* part = reinterpret_cast<long long*>(base + off);
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)s * 4, st);
  if (e != cudaSuccess) return e;
  sparse_rows_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, s, zeta, (uint32_t)seed,
                                                                  (uint32_t)(seed >> 32), table, counts);
  sparse_grid_kernel<<<1, 1024, 0, st>>>(cmax_bits, ncols, counts, s, qexp);
  dim3 grid((unsigned)p.colblocks, (unsigned)p.splits);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t ee = allow_dyn_smem(kern, p.smem);
    if (ee != cudaSuccess) return ee;
    kern<<<grid, kSpThreads, p.smem, st>>>(A, lda, b, m, n, s, zeta, table, qexp, part, p.rows_per_split);
    return cudaGetLastError();
  };
  if (p.cb == 4) e = go(sparse_sketch_kernel<4>);
  else if (p.cb == 2) e = go(sparse_sketch_kernel<2>);
  else e = go(sparse_sketch_kernel<1>);
  if (e != cudaSuccess) return e;
  const int64_t total = ncols * s;
  sparse_finalize_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, p.splits, ncols, s, qexp,
                                                                          1.0 / sqrt((double)zeta), Y);
  return cudaGetLastError();
}

}  // namespace lsq
