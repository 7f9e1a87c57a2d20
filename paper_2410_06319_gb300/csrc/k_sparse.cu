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
//  * quantize kernel: [A | b] rounded once onto the column grids (round half even on the
//    grid, integer arithmetic on the FP64 bits) into an int64 copy.
//  * lists: an exclusive scan of the counts and a fill give, for every sketch row, the
//    list of its (data row, sign) entries (a counting sort; the order within a list is
//    whatever the atomics give, which the exact integer sums make irrelevant).
//  * gather kernel: one CTA per sketch row adds (or subtracts) the int64 rows of its list,
//    threads over the columns (coalesced rows), and writes the row of Y: the exact sum
//    converted once to FP64, times 2^-q_c and zeta^-1/2 (the same operations as the
//    definition, so Y is exact).
// HBM: [A | b] read once and its int64 copy written once, then every data row of the copy
// read zeta times (once per sketch row it lands in); no atomics on the data.
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

// Aq[j][c] = round(a_jc 2^q_c) for c < n, Aq[j][n] = round(b_j 2^q_n); rows of ncols int64.
__global__ void __launch_bounds__(256)
    sparse_quant_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ b, int64_t m,
                        int64_t n, const int* __restrict__ qexp, long long* __restrict__ Aq, int rows_per_cta) {
  const uint64_t* Au = reinterpret_cast<const uint64_t*>(A);
  const uint64_t* bu = reinterpret_cast<const uint64_t*>(b);
  const int64_t ncols = n + 1;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
  for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
    const int q = qexp[c];
    for (int64_t j = r0; j < r1; ++j) {
      const uint64_t u = c < n ? __ldcs(Au + j * lda + c) : bu[j];
      Aq[j * ncols + c] = to_grid(u, q);
    }
  }
}

// offsets = exclusive prefix sums of counts (s + 1 entries; one CTA of 1024 threads, s <= 16384)
__global__ void __launch_bounds__(1024) sparse_scan_kernel(const unsigned* __restrict__ counts, int s,
                                                           unsigned long long* __restrict__ offsets) {
  __shared__ unsigned long long part[1024];
  const int per = (s + 1023) / 1024;
  const int i0 = threadIdx.x * per, i1 = min(s, i0 + per);
  unsigned long long v = 0;
  for (int i = i0; i < i1; ++i) v += counts[i];
  part[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan of the chunk sums (Hillis-Steele)
    const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0ull;
  for (int i = i0; i < i1; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == 1023) offsets[s] = part[1023];
}

// list[offsets[r] + slot] = j | sign << 63 for every entry (j, k) of the row table
__global__ void sparse_fill_kernel(const uint16_t* __restrict__ table, int64_t m, int zeta,
                                   const unsigned long long* __restrict__ offsets, unsigned* __restrict__ cursor,
                                   unsigned long long* __restrict__ list) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m) return;
  for (int k = 0; k < zeta; ++k) {
    const uint16_t tv = table[j * kSpMaxZeta + k];
    const int r = tv & 0x7FFF;
    const unsigned slot = atomicAdd(cursor + r, 1u);
    list[offsets[r] + slot] = (unsigned long long)j | ((unsigned long long)(tv >> 15) << 63);
  }
}

// Y[c][r] = 2^-q_c zeta^-1/2 sum over the list of r of +-Aq[j][c]; one CTA per sketch row r
constexpr int kSpGatherThreads = 256;
constexpr int kSpGatherPer = 5;        // columns per thread: ncols <= 1280
__global__ void __launch_bounds__(kSpGatherThreads)
    sparse_gather_kernel(const long long* __restrict__ Aq, int64_t ncols, int s,
                         const unsigned long long* __restrict__ offsets, const unsigned long long* __restrict__ list,
                         const int* __restrict__ qexp, double scale, double* __restrict__ Y) {
  const int r = blockIdx.x;
  const unsigned long long e0 = offsets[r], e1 = offsets[r + 1];
  long long acc[kSpGatherPer];
#pragma unroll
  for (int i = 0; i < kSpGatherPer; ++i) acc[i] = 0;
  unsigned long long e = e0;
  for (; e + 4 <= e1; e += 4) {      // four rows in flight per thread
    unsigned long long w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = __ldg(list + e + u);
    long long v[4][kSpGatherPer];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long* row = Aq + (int64_t)(w[u] & 0x7FFFFFFFFFFFFFFFull) * ncols;
#pragma unroll
      for (int i = 0; i < kSpGatherPer; ++i) {
        const int64_t c = threadIdx.x + (int64_t)i * kSpGatherThreads;
        v[u][i] = c < ncols ? __ldcs(row + c) : 0ll;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kSpGatherPer; ++i) acc[i] += (w[u] >> 63) ? -v[u][i] : v[u][i];
  }
  for (; e < e1; ++e) {
    const unsigned long long w = __ldg(list + e);
    const long long* row = Aq + (int64_t)(w & 0x7FFFFFFFFFFFFFFFull) * ncols;
#pragma unroll
    for (int i = 0; i < kSpGatherPer; ++i) {
      const int64_t c = threadIdx.x + (int64_t)i * kSpGatherThreads;
      const long long v = c < ncols ? __ldcs(row + c) : 0ll;
      acc[i] += (w >> 63) ? -v : v;
    }
  }
#pragma unroll
  for (int i = 0; i < kSpGatherPer; ++i) {
    const int64_t c = threadIdx.x + (int64_t)i * kSpGatherThreads;
    if (c < ncols) Y[c * s + r] = ldexp((double)acc[i], -qexp[c]) * scale;
  }
}

namespace {
size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
}  // namespace

size_t sparse_workspace(int64_t m, int64_t ncols, int s, int /*splits*/) {
  return al256((size_t)m * kSpMaxZeta * 2) + al256((size_t)s * 4) + al256((size_t)ncols * 4) +
         al256((size_t)(s + 1) * 8) + al256((size_t)s * 4) + al256((size_t)m * kSpMaxZeta * 8) +
         al256((size_t)m * (size_t)ncols * 8) + 1024;
}

SparsePlan plan_sparse(int64_t m, int64_t ncols, int s, int /*num_sms*/) {
  SparsePlan p{};
  p.cb = (int)ncols;          // one gather CTA covers every column of a sketch row
  p.colblocks = 1;
  p.splits = 1;
  p.rows_per_split = m;
  p.smem = 0;
  (void)s;
  return p;
}

cudaError_t launch_sparse_sketch(const SparsePlan& p, const double* A, int64_t lda, const double* b, int64_t m,
                                 int64_t n, int s, int zeta, uint64_t seed,
                                 const unsigned long long* cmax_bits, void* work, double* Y, cudaStream_t st) {
  (void)p;
  if (zeta < 1 || zeta > kSpMaxZeta || zeta > s || s > 16384) return cudaErrorInvalidValue;
  const int64_t ncols = n + 1;
  if (ncols > (int64_t)kSpGatherThreads * kSpGatherPer) return cudaErrorInvalidValue;
  auto* base = static_cast<unsigned char*>(work);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = base + off;
    off += al256(bytes);
    return q;
  };
  auto* table = reinterpret_cast<uint16_t*>(take((size_t)m * kSpMaxZeta * 2));
  auto* counts = reinterpret_cast<unsigned*>(take((size_t)s * 4));
  auto* qexp = reinterpret_cast<int*>(take((size_t)ncols * 4));
  auto* offsets = reinterpret_cast<unsigned long long*>(take((size_t)(s + 1) * 8));
  auto* cursor = reinterpret_cast<unsigned*>(take((size_t)s * 4));
  auto* list = reinterpret_cast<unsigned long long*>(take((size_t)m * kSpMaxZeta * 8));
  auto* Aq = reinterpret_cast<long long*>(take((size_t)m * (size_t)ncols * 8));
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)s * 4, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, (size_t)s * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned row_ctas = (unsigned)((m + 255) / 256);
  sparse_rows_kernel<<<row_ctas, 256, 0, st>>>(m, s, zeta, (uint32_t)seed, (uint32_t)(seed >> 32), table, counts);
  sparse_grid_kernel<<<1, 1024, 0, st>>>(cmax_bits, ncols, counts, s, qexp);
  constexpr int kRows = 16;
  sparse_quant_kernel<<<(unsigned)((m + kRows - 1) / kRows), 256, 0, st>>>(A, lda, b, m, n, qexp, Aq, kRows);
  sparse_scan_kernel<<<1, 1024, 0, st>>>(counts, s, offsets);
  sparse_fill_kernel<<<row_ctas, 256, 0, st>>>(table, m, zeta, offsets, cursor, list);
  sparse_gather_kernel<<<(unsigned)s, kSpGatherThreads, 0, st>>>(Aq, ncols, s, offsets, list, qexp,
                                                                 1.0 / sqrt((double)zeta), Y);
  return cudaGetLastError();
}

}  // namespace lsq
