// Streaming passes over A and the small kernels of LSQR and FGMRES (Alg. 2).
//
// Passes (one coalesced, 128-bit vectorised read of A per call, a warp per
// row, the row kept in registers for both products):
//   LSQR (Alg. 2, LSQR start):  q = A t + cu u ; P = A^T q ; sum q^2
//   FGMRES (Alg. 2, FGMRES):  w_top = v_top + A z_bot ; P = A^T v_top
//   residual (refinement, u_r):  f = b - r - A x ; P = A^T (-r)
// P is reduced per CTA (fixed order) and then across CTAs by colsum, so the
// results are deterministic.
#include <type_traits>

#include <algorithm>

#include "common.cuh"
#include "batch.h"
#include "iter.h"
#include "kernels.h"
#include "trsv.cuh"

namespace lsq {

// ============================================================ block helpers
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  return red[32];
}


template <typename T, int VW>
struct VecOf;
template <>
struct VecOf<float, 4> {
  using type = float4;
};
template <>
struct VecOf<double, 2> {
  using type = double2;
};
template <>
struct VecOf<double, 1> {
  using type = double;
};

template <typename T, int VW>
__device__ __forceinline__ void load_vec(const T* p, T (&o)[VW], bool streaming) {
  using V = typename VecOf<T, VW>::type;
  V v = streaming ? __ldcs(reinterpret_cast<const V*>(p)) : *reinterpret_cast<const V*>(p);
  const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int k = 0; k < VW; ++k) o[k] = e[k];
}

template <typename T, int VW, int VPL, int MODE>
__device__ __forceinline__ void pass_body(PassArgs<T> p, int64_t blk, int64_t nblk) {
  if (p.done && *p.done) return;
  if (p.jp) {
    const int64_t j = *p.jp;
    p.x += j * p.xstr;
    p.v += j * p.vstr;
  }
  extern __shared__ __align__(16) unsigned char pass_smem[];
  T* red = reinterpret_cast<T*>(pass_smem);          // [8 warps][nv * VW]
  __shared__ double sqred[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = blk * 8 + warp, tw = nblk * 8;
  T xv[VPL][VW], acc[VPL][VW];
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int idx = lane + 32 * v;
    if (idx < p.nv) {
      load_vec<T, VW>(p.x + (int64_t)idx * VW, xv[v], false);
    } else {
      for (int k = 0; k < VW; ++k) xv[v][k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < VW; ++k) acc[v][k] = T(0);
  }
  T cu = T(0);
  if (MODE == PM_LSQR) cu = (T)((p.cu_ptr ? *p.cu_ptr : 1.0) * p.cu_mul);
  double sqacc = 0.0;
  for (int64_t i = gw; i < p.m; i += 2 * tw) {
    const int64_t i2 = i + tw;
    const bool has2 = i2 < p.m;
    T a[VPL][VW], a2[VPL][VW];
    const T* row = p.A + i * p.lda;
    const T* row2 = p.A + i2 * p.lda;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int idx = lane + 32 * v;
      if (idx < p.nv) {
        load_vec<T, VW>(row + (int64_t)idx * VW, a[v], true);
      } else {
        for (int k = 0; k < VW; ++k) a[v][k] = T(0);
      }
      if (has2 && idx < p.nv) {
        load_vec<T, VW>(row2 + (int64_t)idx * VW, a2[v], true);
      } else {
        for (int k = 0; k < VW; ++k) a2[v][k] = T(0);
      }
    }
    T d = 0, d2 = 0;
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        d = fma(a[v][k], xv[v][k], d);
        d2 = fma(a2[v][k], xv[v][k], d2);
      }
    warp_sum2(d, d2);
    T c1, c2 = T(0);
    if (MODE == PM_LSQR) {
      const T q = d + cu * p.uin[i];
      c1 = q;
      if (lane == 0) {
        p.uout[i] = q;
        sqacc += (double)q * (double)q;
      }
      if (has2) {
        const T q2 = d2 + cu * p.uin[i2];
        c2 = q2;
        if (lane == 0) {
          p.uout[i2] = q2;
          sqacc += (double)q2 * (double)q2;
        }
      }
    } else if (MODE == PM_FGM) {
      c1 = p.v[i];
      if (lane == 0) p.az[i] = d;
      if (has2) {
        c2 = p.v[i2];
        if (lane == 0) p.az[i2] = d2;
      }
    } else {
      const double ri = p.r[i];
      c1 = (T)(-ri);
      if (lane == 0) p.f[i] = (p.b[i] - ri) - (double)d;
      if (has2) {
        const double ri2 = p.r[i2];
        c2 = (T)(-ri2);
        if (lane == 0) p.f[i2] = (p.b[i2] - ri2) - (double)d2;
      }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
      for (int k = 0; k < VW; ++k) acc[v][k] = fma(c1, a[v][k], fma(c2, a2[v][k], acc[v][k]));
  }
  // CTA reduction of acc (fixed order over warps)
  const int width = p.nv * VW;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int idx = lane + 32 * v;
    if (idx < p.nv) {
      for (int k = 0; k < VW; ++k) red[warp * width + idx * VW + k] = acc[v][k];
    }
  }
  if (MODE == PM_LSQR && lane == 0) sqred[warp] = sqacc;
  __syncthreads();
  for (int c = threadIdx.x; c < p.n; c += blockDim.x) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += red[w * width + c];
    p.Pblk[blk * p.n + c] = s;
  }
  if (MODE == PM_LSQR && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sqred[w];
    p.sq[blk] = s;
  }
}

template <typename T, int VW, int VPL, int MODE>
__global__ void __launch_bounds__(256) pass_kernel(PassArgs<T> p) {
  pass_body<T, VW, VPL, MODE>(p, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------ bulk-streamed passes
// A producer warp streams stages of 8 consecutive rows of A into a shared-memory
// ring with cp.async.bulk (completion on an mbarrier); eight consumer warps take
// one row of each stage.  Each CTA owns a contiguous range of rows.  The per-row
// scalars of the next stage are loaded one stage ahead.
//   PM_LSQR: q = A t + cu u ; u_out = q ; P = A^T q ; sq = sum q^2
//   PM_FGM : az = A z ; P = A^T v            (v_top + az is formed by the Arnoldi step)
//   PM_RES : f = b - r - A x ; P = A^T (-r)
constexpr int kBulkRows = 16;
constexpr int kBulkThreads = (kBulkRows + 1) * 32;

template <typename T>
struct BulkArgs {
  const T* A;
  int64_t lda, m;
  int n, nv, stages;
  int64_t rows_per_cta;
  const T* x;                  // multiplied vector (nv * VW entries, zero padded)
  const int* jp;               // FGM: x and v are column (*jp) of their bases
  int64_t xstr, vstr;
  const T* uin;                // LSQR
  T* uout;
  const double* cu_ptr;
  double cu_mul;
  const T* v;                  // FGM coefficient vector
  T* az;
  const double* r;             // RES
  const double* b;
  double* f;
  T* Pblk;
  double* sq;
  const int* done;
  int* err;
};

template <typename T, int VW, int VPL, int MODE>
__global__ void __launch_bounds__(kBulkThreads, 1) pass_bulk_kernel(BulkArgs<T> p) {
  if (p.done && *p.done) return;
  if (MODE == PM_FGM && p.jp) {
    const int64_t j = *p.jp;
    p.x += j * p.xstr;
    p.v += j * p.vstr;
  }
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  const uint32_t stage_bytes = (uint32_t)(kBulkRows * p.lda * sizeof(T));
  uint64_t* bars = reinterpret_cast<uint64_t*>(bulk_smem + (size_t)p.stages * stage_bytes);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + p.stages);
  __shared__ double sqred[kBulkRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * p.rows_per_cta;
  const int64_t r1 = min(p.m, r0 + p.rows_per_cta);
  const int nst = r0 < r1 ? (int)((r1 - r0 + kBulkRows - 1) / kBulkRows) : 0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < p.stages; ++k) {
      mbar_init(full0 + 8 * k, 1);
      mbar_init(empty0 + 8 * k, kBulkRows);
    }
    fence_barrier_init();
  }
  __syncthreads();
  T acc[VPL][VW];
#pragma unroll
  for (int v = 0; v < VPL; ++v)
#pragma unroll
    for (int k = 0; k < VW; ++k) acc[v][k] = T(0);
  float sqacc = 0.f;
  if (warp == kBulkRows) {
    // ---------------- producer
    if (lane == 0) {
      const uint64_t pol = l2_policy_evict_first();   // A is read once per pass
      for (int it = 0; it < nst; ++it) {
        const int slot = it % p.stages;
        const uint32_t ph = (uint32_t)(it / p.stages) & 1u;
        if (!mbar_wait(empty0 + 8 * slot, ph ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) break;
        const int64_t row0 = r0 + (int64_t)it * kBulkRows;
        const int rows = (int)min((int64_t)kBulkRows, r1 - row0);
        const uint32_t bytes = (uint32_t)(rows * p.lda * sizeof(T));
        mbar_arrive_expect_tx(full0 + 8 * slot, bytes);
        bulk_load_hint(smem_u32(bulk_smem + (size_t)slot * stage_bytes), p.A + row0 * p.lda, bytes,
                       full0 + 8 * slot, pol);
      }
    }
  } else {
    // ---------------- consumers: warp `warp` takes row `warp` of every stage
    T xv[VPL][VW];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int idx = lane + 32 * v;
      if (idx < p.nv) {
        load_vec<T, VW>(p.x + (int64_t)idx * VW, xv[v], false);
      } else {
        for (int k = 0; k < VW; ++k) xv[v][k] = T(0);
      }
    }
    const T cu = (MODE == PM_LSQR) ? (T)((p.cu_ptr ? *p.cu_ptr : 1.0) * p.cu_mul) : T(0);
    // per-row scalars for a window of 32 stages: lane l holds the scalars of stage
    // base + l; the next window is loaded while the current one is consumed
    // scalars in the pass precision (no FP64 conversions in the FP32 passes)
    using S = typename std::conditional<MODE == PM_RES, double, T>::type;
    auto load_window = [&](int base, S& s0, S& s1) {
      const int it = base + lane;
      const int64_t row = r0 + (int64_t)it * kBulkRows + warp;
      s0 = S(0);
      s1 = S(0);
      if (it < nst && row < r1) {
        if constexpr (MODE == PM_LSQR) s0 = p.uin[row];
        if constexpr (MODE == PM_FGM) s0 = p.v[row];
        if constexpr (MODE == PM_RES) {
          s0 = p.r[row];
          s1 = p.b[row];
        }
      }
    };
    S w0, w1, x0n, x1n;
    load_window(0, w0, w1);
    load_window(32, x0n, x1n);
    for (int it = 0; it < nst; ++it) {
      if ((it & 31) == 0 && it > 0) {
        w0 = x0n;
        w1 = x1n;
        load_window(it + 32, x0n, x1n);
      }
      const S c0 = __shfl_sync(0xffffffffu, w0, it & 31);
      const S c1s = (MODE == PM_RES) ? __shfl_sync(0xffffffffu, w1, it & 31) : S(0);
      const int slot = it % p.stages;
      const uint32_t ph = (uint32_t)(it / p.stages) & 1u;
      if (!mbar_wait(full0 + 8 * slot, ph, p.err, DEV_TIMEOUT_FULL)) break;
      const int64_t row = r0 + (int64_t)it * kBulkRows + warp;
      if (row < r1) {
        const T* srow = reinterpret_cast<const T*>(bulk_smem + (size_t)slot * stage_bytes) + warp * p.lda;
        T a[VPL][VW];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const int idx = lane + 32 * v;
          if (idx < p.nv) {
            load_vec<T, VW>(srow + idx * VW, a[v], false);
          } else {
            for (int k = 0; k < VW; ++k) a[v][k] = T(0);
          }
        }
        // four interleaved chains: in LSQR the row's A^T q update waits on this sum
        T dq[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
          for (int k = 0; k < VW; ++k) dq[(v * VW + k) & 3] = fma(a[v][k], xv[v][k], dq[(v * VW + k) & 3]);
        T d = (dq[0] + dq[1]) + (dq[2] + dq[3]);
        d = warp_sum(d);
        T coef;
        if (MODE == PM_LSQR) {
          const T q = d + cu * (T)c0;
          coef = q;
          if (lane == 0) {
            p.uout[row] = q;
            sqacc = fmaf((float)q, (float)q, sqacc);
          }
        } else if (MODE == PM_FGM) {
          coef = (T)c0;
          if (lane == 0) p.az[row] = d;
        } else {
          coef = (T)(-c0);
          if (lane == 0) p.f[row] = (c1s - c0) - (double)d;
        }
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
          for (int k = 0; k < VW; ++k) acc[v][k] = fma(coef, a[v][k], acc[v][k]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * slot);
    }
  }
  __syncthreads();   // every stage consumed: the ring is free for the reduction
  const int width = p.nv * VW;
  T* red = reinterpret_cast<T*>(bulk_smem);
  if (warp < kBulkRows) {
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int idx = lane + 32 * v;
      if (idx < p.nv) {
        for (int k = 0; k < VW; ++k) red[warp * width + idx * VW + k] = acc[v][k];
      }
    }
    if (MODE == PM_LSQR && lane == 0) sqred[warp] = (double)sqacc;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < p.n; c += blockDim.x) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < kBulkRows; ++w) s += red[w * width + c];
    p.Pblk[(int64_t)blockIdx.x * p.n + c] = s;
  }
  if (MODE == PM_LSQR && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBulkRows; ++w) s += sqred[w];
    p.sq[blockIdx.x] = s;
  }
}

int bulk_blocks(int num_sms) { return num_sms; }

template <typename T, int VW, int MODE>
static cudaError_t dispatch_bulk(BulkArgs<T> p, int nblk, int num_sms_unused, cudaStream_t st) {
  const int vpl = (p.nv + 31) / 32;
  const size_t stage_bytes = (size_t)kBulkRows * p.lda * sizeof(T);
  const size_t budget = 200 * 1024;
  int stages = (int)(budget / stage_bytes);
  if (stages > 12) stages = 12;
  if (stages < 2) return cudaErrorInvalidValue;
  p.stages = stages;
  p.rows_per_cta = ((p.m + nblk - 1) / nblk + kBulkRows - 1) / kBulkRows * kBulkRows;
  const size_t red_bytes = (size_t)kBulkRows * p.nv * VW * sizeof(T);
  size_t smem = (size_t)stages * stage_bytes;
  if (smem < red_bytes) smem = red_bytes;
  smem += 2 * stages * 8;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<nblk, kBulkThreads, smem, st>>>(p);
    return cudaGetLastError();
  };
  if (vpl <= 1) return go(pass_bulk_kernel<T, VW, 1, MODE>);
  if (vpl <= 2) return go(pass_bulk_kernel<T, VW, 2, MODE>);
  if (vpl <= 4) return go(pass_bulk_kernel<T, VW, 4, MODE>);
  if (vpl <= 8) return go(pass_bulk_kernel<T, VW, 8, MODE>);
  if constexpr (VW <= 2) {
    if (vpl <= 16) return go(pass_bulk_kernel<T, VW, 16, MODE>);
  }
  return cudaErrorInvalidValue;
}

int pass_blocks(int num_sms) { return num_sms; }

template <typename T, int VW, int MODE>
static cudaError_t dispatch_pass(const PassArgs<T>& p, int nblk, cudaStream_t st) {
  const int vpl = (p.nv + 31) / 32;
  const size_t smem = (size_t)8 * p.nv * VW * sizeof(T);
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = allow_dyn_smem(kern, smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<nblk, 256, smem, st>>>(p);
    return cudaGetLastError();
  };
  if (vpl <= 1) return go(pass_kernel<T, VW, 1, MODE>);
  if (vpl <= 2) return go(pass_kernel<T, VW, 2, MODE>);
  if (vpl <= 4) return go(pass_kernel<T, VW, 4, MODE>);
  if (vpl <= 8) return go(pass_kernel<T, VW, 8, MODE>);
  if constexpr (VW <= 2) {
    if (vpl <= 16) return go(pass_kernel<T, VW, 16, MODE>);
  }
  if constexpr (VW == 1) {
    if (vpl <= 32) return go(pass_kernel<T, VW, 32, MODE>);
  }
  return cudaErrorInvalidValue;
}

// Vector width for an FP64 matrix: double2 when rows and the base are 16-byte aligned.
static int f64_vw(const double* A, int64_t lda, int64_t n) {
  return ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda % 2) == 0 && (n % 2) == 0) ? 2 : 1;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// The bulk-streamed ring needs two stages of kBulkRows rows within its 200 KB of
// shared memory and a bulk instantiation for the row's vector count; wider rows
// (FP64 beyond 800 columns) take the register-blocked pass kernel instead.
template <typename T, int VW>
static bool bulk_fits(int64_t lda, int64_t nv) {
  const int64_t vpl = (nv + 31) / 32;
  return 2 * (size_t)kBulkRows * (size_t)lda * sizeof(T) <= (size_t)200 * 1024 &&
         (vpl <= 8 || (VW <= 2 && vpl <= 16));
}

template <typename T>
cudaError_t launch_pass_lsqr_t(const T* A, int64_t lda, int64_t m, int64_t n, const T* t,
                               const T* u_in, const double* cu_ptr, double cu_mul, T* u_out, T* Pblk,
                               double* sq, int nblk, const int* done, cudaStream_t st) {
  int vw = 4;
  bool bulk = aligned16(A);
  if constexpr (sizeof(T) == 4) {
    bulk = bulk && bulk_fits<float, 4>(lda, (lda + 3) / 4);
  } else {
    vw = f64_vw(A, lda, n);
    bulk = bulk && lda % 2 == 0 &&
           (vw == 2 ? bulk_fits<double, 2>(lda, n / 2) : bulk_fits<double, 1>(lda, n));
  }
  if (bulk) {
    BulkArgs<T> b{};
    b.A = A; b.lda = lda; b.m = m; b.n = (int)n;
    b.x = t; b.uin = u_in; b.uout = u_out; b.cu_ptr = cu_ptr; b.cu_mul = cu_mul;
    b.Pblk = Pblk; b.sq = sq; b.done = done;
    if constexpr (sizeof(T) == 4) {
      b.nv = (int)((lda + 3) / 4);
      return dispatch_bulk<float, 4, PM_LSQR>(b, nblk, 0, st);
    } else {
      if (vw == 2) {
        b.nv = (int)(n / 2);
        return dispatch_bulk<double, 2, PM_LSQR>(b, nblk, 0, st);
      }
      b.nv = (int)n;
      return dispatch_bulk<double, 1, PM_LSQR>(b, nblk, 0, st);
    }
  }
  PassArgs<T> p{};
  p.A = A; p.lda = lda; p.m = m; p.n = (int)n;
  p.x = t; p.uin = u_in; p.uout = u_out; p.cu_ptr = cu_ptr; p.cu_mul = cu_mul;
  p.Pblk = Pblk; p.sq = sq; p.done = done;
  if constexpr (sizeof(T) == 4) {
    p.nv = (int)((lda + 3) / 4);   // A32 rows are zero padded to lda (a multiple of 4)
    return dispatch_pass<float, 4, PM_LSQR>(p, nblk, st);
  } else {
    if (vw == 2) {
      p.nv = (int)(n / 2);
      return dispatch_pass<double, 2, PM_LSQR>(p, nblk, st);
    }
    p.nv = (int)n;
    return dispatch_pass<double, 1, PM_LSQR>(p, nblk, st);
  }
}


template <typename TA>
cudaError_t launch_pass_fgm(const TA* A, int64_t lda, int64_t m, int64_t n, const TA* z,
                            const TA* v, TA* az, TA* Pblk, int nblk, const int* done, cudaStream_t st,
                            const int* jp, int64_t zs, int64_t vstr, int* err) {
  BulkArgs<TA> b{};
  b.A = A; b.lda = lda; b.m = m; b.n = (int)n;
  b.x = z; b.v = v; b.az = az; b.Pblk = Pblk; b.done = done; b.err = err;
  b.jp = jp; b.xstr = zs; b.vstr = vstr;
  if constexpr (sizeof(TA) == 4) {
    if (!aligned16(A) || (lda % 4) != 0) return cudaErrorInvalidValue;
    b.nv = (int)((lda + 3) / 4);
    return dispatch_bulk<float, 4, PM_FGM>(b, nblk, 0, st);
  } else {
    const int vw = f64_vw(A, lda, n);
    if (aligned16(A) && (lda % 2) == 0 &&
        (vw == 2 ? bulk_fits<double, 2>(lda, n / 2) : bulk_fits<double, 1>(lda, n))) {
      if (vw == 2) {
        b.nv = (int)(n / 2);
        return dispatch_bulk<double, 2, PM_FGM>(b, nblk, 0, st);
      }
      b.nv = (int)n;
      return dispatch_bulk<double, 1, PM_FGM>(b, nblk, 0, st);
    }
    PassArgs<double> q{};
    q.A = A; q.lda = lda; q.m = m; q.n = (int)n;
    q.x = z; q.v = v; q.az = az; q.Pblk = Pblk; q.done = done;
    q.jp = jp; q.xstr = zs; q.vstr = vstr;
    if (vw == 2) {
      q.nv = (int)(n / 2);
      return dispatch_pass<double, 2, PM_FGM>(q, nblk, st);
    }
    q.nv = (int)n;
    return dispatch_pass<double, 1, PM_FGM>(q, nblk, st);
  }
}
template cudaError_t launch_pass_fgm<float>(const float*, int64_t, int64_t, int64_t, const float*,
                                            const float*, float*, float*, int, const int*,
                                            cudaStream_t, const int*, int64_t, int64_t, int*);
template cudaError_t launch_pass_fgm<double>(const double*, int64_t, int64_t, int64_t, const double*,
                                             const double*, double*, double*, int, const int*,
                                             cudaStream_t, const int*, int64_t, int64_t, int*);

cudaError_t launch_pass_res(const double* A, int64_t lda, int64_t m, int64_t n, const double* x,
                            const double* r, const double* b, double* f, double* Pblk, int nblk,
                            cudaStream_t st) {
  const int vw = f64_vw(A, lda, n);
  if (aligned16(A) && lda % 2 == 0 &&
      (vw == 2 ? bulk_fits<double, 2>(lda, n / 2) : bulk_fits<double, 1>(lda, n))) {
    BulkArgs<double> q{};
    q.A = A; q.lda = lda; q.m = m; q.n = (int)n;
    q.x = x; q.r = r; q.b = b; q.f = f; q.Pblk = Pblk;
    if (f64_vw(A, lda, n) == 2) {
      q.nv = (int)(n / 2);
      return dispatch_bulk<double, 2, PM_RES>(q, nblk, 0, st);
    }
    q.nv = (int)n;
    return dispatch_bulk<double, 1, PM_RES>(q, nblk, 0, st);
  }
  PassArgs<double> p{};
  p.A = A; p.lda = lda; p.m = m; p.n = (int)n;
  p.x = x; p.r = r; p.b = b; p.f = f; p.Pblk = Pblk;
  if (f64_vw(A, lda, n) == 2) {
    p.nv = (int)(n / 2);
    return dispatch_pass<double, 2, PM_RES>(p, nblk, st);
  }
  p.nv = (int)n;
  return dispatch_pass<double, 1, PM_RES>(p, nblk, st);
}

// ------------------------------------------------------------ column sums
template <typename TP, typename TO>
__device__ __forceinline__ void colsum_body(const TP* __restrict__ P, int nblk, int64_t n, const double* scale_ptr,
                                            double scale_mul, TO* __restrict__ out, const int* done, int64_t bx) {
  if (done && *done) return;
  __shared__ double part[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t c = bx * 32 + tx;
  double s = 0.0;
  if (c < n)
    for (int b = ty; b < nblk; b += 32) s += (double)P[(int64_t)b * n + c];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && c < n) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += part[k][tx];
    const double sc = (scale_ptr ? *scale_ptr : 1.0) * scale_mul;
    out[c] = (TO)(t * sc);
  }
}

template <typename TP, typename TO>
__global__ void colsum_kernel(const TP* __restrict__ P, int nblk, int64_t n, const double* scale_ptr,
                              double scale_mul, TO* __restrict__ out, const int* done) {
  colsum_body<TP, TO>(P, nblk, n, scale_ptr, scale_mul, out, done, blockIdx.x);
}

template <typename TP, typename TO>
cudaError_t launch_colsum(const TP* P, int nblk, int64_t n, const double* scale_ptr, double scale_mul,
                          TO* out, const int* done, cudaStream_t st) {
  colsum_kernel<TP, TO><<<(unsigned)((n + 31) / 32), dim3(32, 32), 0, st>>>(P, nblk, n, scale_ptr,
                                                                           scale_mul, out, done);
  return cudaGetLastError();
}
template cudaError_t launch_colsum<float, float>(const float*, int, int64_t, const double*, double,
                                                 float*, const int*, cudaStream_t);
template cudaError_t launch_colsum<double, double>(const double*, int, int64_t, const double*, double,
                                                   double*, const int*, cudaStream_t);
template cudaError_t launch_colsum<double, float>(const double*, int, int64_t, const double*, double,
                                                  float*, const int*, cudaStream_t);
template cudaError_t launch_colsum<float, double>(const float*, int, int64_t, const double*, double,
                                                  double*, const int*, cudaStream_t);

// ============================================================ LSQR kernels
template <typename TP>
cudaError_t launch_pass_lsqr_any(const TP* A, int64_t lda, int64_t m, int64_t n, const TP* t,
                                 const TP* u_in, const double* cu_ptr, double cu_mul, TP* u_out,
                                 TP* Pblk, double* sq, int nblk, const int* done, cudaStream_t st) {
  return launch_pass_lsqr_t<TP>(A, lda, m, n, t, u_in, cu_ptr, cu_mul, u_out, Pblk, sq, nblk, done, st);
}
template cudaError_t launch_pass_lsqr_any<float>(const float*, int64_t, int64_t, int64_t, const float*,
                                                 const float*, const double*, double, float*, float*,
                                                 double*, int, const int*, cudaStream_t);
template cudaError_t launch_pass_lsqr_any<double>(const double*, int64_t, int64_t, int64_t, const double*,
                                                  const double*, const double*, double, double*,
                                                  double*, double*, int, const int*, cudaStream_t);

// ------------------------------------------------------------ fused LSQR step
// beta = ||q|| from the per-CTA sums of squares (every CTA recomputes it);
// out[c] = (A^T q)_c / beta.  Block 0 publishes beta and 1/beta.
template <typename TP>
__device__ __forceinline__ void lsqr_colsum_body(const TP* __restrict__ P, int nblk, int64_t n, const double* sq,
                                                 LsqrState* st, bool init, TP* __restrict__ out, int64_t bx) {
  if (!init && st->done) return;
  __shared__ double part[32][33];
  __shared__ double beta_s;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  double q = 0.0;
  for (int b = tid; b < nblk; b += 1024) q += sq[b];
  q = warp_sum(q);
  if (tx == 0) part[ty][32] = q;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += part[k][32];
    beta_s = sqrt(t);
  }
  __syncthreads();
  const double beta = beta_s;
  const double us = beta > 0.0 ? 1.0 / beta : 0.0;
  if (bx == 0 && tid == 0) {
    st->beta = beta;
    st->us = us;
    if (init) st->phibar = beta;
  }
  const int64_t c = bx * 32 + tx;
  double sacc = 0.0;
  if (c < n)
    for (int b = ty; b < nblk; b += 32) sacc += (double)P[(int64_t)b * n + c];
  part[ty][tx] = sacc;
  __syncthreads();
  if (ty == 0 && c < n) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += part[k][tx];
    out[c] = (TP)(t * us);
  }
}

template <typename TP>
__global__ void lsqr_colsum_kernel(const TP* __restrict__ P, int nblk, int64_t n, const double* sq,
                                   LsqrState* st, bool init, TP* __restrict__ out) {
  lsqr_colsum_body<TP>(P, nblk, n, sq, st, init, out, blockIdx.x);
}

// One CTA: vt = R^-T s ; (init) alpha v = vt, w = v, z = 0 ; (iteration)
// alpha v = vt - beta v, plane rotation, z += (phi/rho) w, w = v - (theta/rho) w,
// stopping tests ; then t = R^-1 v for the next pass.
template <typename T>
__device__ __forceinline__ void lsqr_step_body(const Tri<T>& f, const T* __restrict__ s, T* __restrict__ v,
                                               T* __restrict__ w, T* __restrict__ z, T* __restrict__ t,
                                               LsqrState* st, bool init) {
  if (!init && st->done) return;
  __shared__ T xs[1024];
  __shared__ double red[33];
  __shared__ double coef[3];
  extern __shared__ __align__(16) unsigned char step_buf[];
  const int n = (int)f.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = s[i];
  __syncthreads();
  if (!block_trsv<T, false>(f.L, f.ld, f.DL, n, xs, step_buf, f.err)) return;   // xs = R^-T s
  const double beta = st->beta;
  double ss = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T vv = init ? xs[i] : xs[i] - (T)beta * v[i];
    ss += (double)vv * (double)vv;
  }
  ss = block_sum_d(ss, red);
  const double alpha = sqrt(ss);
  if (threadIdx.x == 0) {
    if (init) {
      st->alpha = alpha;
      st->rhobar = alpha;
      st->anorm2 = 0.0;
      st->its = 0;
      st->normr = beta;
      st->normar = alpha * beta;
      st->normA = 0.0;
      st->flag = (beta == 0.0 || alpha == 0.0) ? 3 : 0;
      st->done = (st->flag != 0 || st->maxit <= 0) ? 1 : 0;
      coef[0] = 0.0;
      coef[1] = 0.0;
    } else {
      const double alpha_old = st->alpha;
      const double anorm2 = st->anorm2 + alpha_old * alpha_old + beta * beta;
      const double rhobar = st->rhobar;
      const double rho = sqrt(rhobar * rhobar + beta * beta);
      const double c = rhobar / rho, sn = beta / rho;
      const double theta = sn * alpha;
      const double phi = c * st->phibar;
      const double phibar = sn * st->phibar;
      coef[0] = phi / rho;
      coef[1] = theta / rho;
      st->rhobar = -c * alpha;
      st->phibar = phibar;
      st->anorm2 = anorm2;
      st->alpha = alpha;
      st->its += 1;
      st->normr = fabs(phibar);
      st->normar = fabs(phibar * alpha * c);
      st->normA = sqrt(anorm2);
      int flag = 0;
      if (st->normr <= st->tol * st->normb) flag = 1;
      else if (st->normar <= st->tol * st->normA * st->normr) flag = 2;
      else if (beta == 0.0 || alpha == 0.0) flag = 3;
      st->flag = flag;
      st->done = (flag != 0 || st->its >= st->maxit) ? 1 : 0;
    }
    st->cu = -alpha * st->us;
  }
  __syncthreads();
  const T ia = alpha > 0.0 ? (T)(1.0 / alpha) : T(0);
  const T c0 = (T)coef[0], c1 = (T)coef[1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T vn = (init ? xs[i] : xs[i] - (T)beta * v[i]) * ia;
    if (init) {
      w[i] = vn;
      z[i] = T(0);
    } else {
      const T wi = w[i];
      z[i] = z[i] + c0 * wi;
      w[i] = vn - c1 * wi;
    }
    v[i] = vn;
    xs[i] = vn;
  }
  __syncthreads();
  if (!block_trsv<T, true>(f.R, f.ld, f.DU, n, xs, step_buf, f.err)) return;    // t = R^-1 v
  for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = xs[i];
}

template <typename T>
__global__ void __launch_bounds__(kTrsvThreads)
    lsqr_step_kernel(Tri<T> f, const T* __restrict__ s, T* __restrict__ v, T* __restrict__ w,
                     T* __restrict__ z, T* __restrict__ t, LsqrState* st, bool init) {
  lsqr_step_body<T>(f, s, v, w, z, t, st, init);
}

template <typename T>
cudaError_t launch_lsqr_colsum(const T* P, int nblk, int64_t n, const double* sq, LsqrState* st,
                               bool init, T* out, cudaStream_t s) {
  lsqr_colsum_kernel<T><<<(unsigned)((n + 31) / 32), dim3(32, 32), 0, s>>>(P, nblk, n, sq, st, init, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_lsqr_step(const Tri<T>& f, const T* s, T* v, T* w, T* z, T* t, LsqrState* st,
                             bool init, cudaStream_t strm) {
  if (f.n > 1024) return cudaErrorInvalidValue;
  const size_t smem = TrsvSmem<T>::bytes;
  cudaError_t e = allow_dyn_smem(lsqr_step_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  lsqr_step_kernel<T><<<1, kTrsvThreads, smem, strm>>>(f, s, v, w, z, t, st, init);
  return cudaGetLastError();
}
template cudaError_t launch_lsqr_colsum<float>(const float*, int, int64_t, const double*, LsqrState*, bool, float*, cudaStream_t);
template cudaError_t launch_lsqr_colsum<double>(const double*, int, int64_t, const double*, LsqrState*, bool, double*, cudaStream_t);
template cudaError_t launch_lsqr_step<float>(const Tri<float>&, const float*, float*, float*, float*, float*, LsqrState*, bool, cudaStream_t);
template cudaError_t launch_lsqr_step<double>(const Tri<double>&, const double*, double*, double*, double*, double*, LsqrState*, bool, cudaStream_t);

// ============================================================ vector kernels
// out[i] = x[i] * a + y[i] * b  (types converted), i < len
template <typename TX, typename TY, typename TO>
__global__ void axpby_kernel(const TX* x, double a, const TY* y, double b, TO* out, int64_t len) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= len) return;
  double v = (double)x[i] * a;
  if (y) v += (double)y[i] * b;
  out[i] = (TO)v;
}

template <typename TX, typename TY, typename TO>
cudaError_t launch_axpby(const TX* x, double a, const TY* y, double b, TO* out, int64_t len,
                         cudaStream_t st) {
  if (len <= 0) return cudaSuccess;
  axpby_kernel<TX, TY, TO><<<(unsigned)((len + 255) / 256), 256, 0, st>>>(x, a, y, b, out, len);
  return cudaGetLastError();
}
template cudaError_t launch_axpby<double, double, float>(const double*, double, const double*, double, float*, int64_t, cudaStream_t);
template cudaError_t launch_axpby<double, double, double>(const double*, double, const double*, double, double*, int64_t, cudaStream_t);
template cudaError_t launch_axpby<float, double, double>(const float*, double, const double*, double, double*, int64_t, cudaStream_t);
template cudaError_t launch_axpby<double, float, double>(const double*, double, const float*, double, double*, int64_t, cudaStream_t);
template cudaError_t launch_axpby<float, float, double>(const float*, double, const float*, double, double*, int64_t, cudaStream_t);
template cudaError_t launch_axpby<float, float, float>(const float*, double, const float*, double, float*, int64_t, cudaStream_t);

// partial[b] = sum over the block's range of x_i * y_i (x, y double; y = x for norms)
__global__ void dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   int64_t len, double* partial) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void sum_partials_kernel(const double* partial, int nblk, double* out, bool take_sqrt) {
  __shared__ double red[33];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : s;
}

cudaError_t launch_dot(const double* x, const double* y, int64_t len, double* partial, int nblk,
                       double* out, bool take_sqrt, cudaStream_t st) {
  dot_partial_kernel<<<nblk, 256, 0, st>>>(x, y, len, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<1, 1024, 0, st>>>(partial, nblk, out, take_sqrt);
  return cudaGetLastError();
}

// ============================================================ FGMRES kernels
// V column-major with leading dimension ld = m + n; H column-major (maxit+1 rows).
__global__ void gm_init_kernel(const double* sq_partial, int nblk, GmState* st, double* g) {
  __shared__ double red[33];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += sq_partial[b];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    const double beta = sqrt(s);
    st->beta0 = beta;
    st->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
    st->j = 0;
    st->relres = beta > 0.0 ? 1.0 : 0.0;
    st->done = (beta == 0.0 || st->maxit <= 0) ? 1 : 0;
    g[0] = beta;
  }
}

// h_{j+1,j} = sqrt(s); Givens rotations on column j; residual estimate; j++.
// One warp (warp 0 of block 0 of the Arnoldi step), with the unrotated column h_{0..j, j}
// in shared memory (hcol, rotated in place): the other warps of the block keep working.
__device__ void gm_finish_warp(double s, GmState* st, double* hcol, double* H, int ldh, double* cs,
                               double* sn, double* g) {
  __shared__ double css[130], sns[130];
  const int lane = threadIdx.x & 31;
  const int j = st->j;
  for (int i = lane; i < j; i += 32) {
    css[i] = cs[i];
    sns[i] = sn[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double hn = sqrt(s);
    hcol[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = css[i] * hcol[i] + sns[i] * hcol[i + 1];
      hcol[i + 1] = -sns[i] * hcol[i] + css[i] * hcol[i + 1];
      hcol[i] = t;
    }
    const double den = hypot(hcol[j], hcol[j + 1]);
    cs[j] = den > 0.0 ? hcol[j] / den : 1.0;
    sn[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
    hcol[j] = den;
    hcol[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    st->relres = fabs(g[j + 1]) / st->beta0;
    st->inv_h = hn > 0.0 ? 1.0 / hn : 0.0;
    st->j = j + 1;
    st->done = (st->relres <= st->tol || st->j >= st->maxit || hn == 0.0) ? 1 : 0;
  }
  __syncwarp();
  double* hc = H + (int64_t)j * ldh;
  for (int i = lane; i <= j + 1; i += 32) hc[i] = hcol[i];
}

// ---------------------------------------------------------------- fused Arnoldi step
// One cooperative launch per FGMRES iteration, one 512-thread CTA per SM, each owning a
// contiguous row range of the length-(m+n) vectors; FP64 throughout.
//   w_top = v_top + A z; partials of h = V^T w and of ||w||^2 (eight basis columns per
//   sweep over the rows, so w is read once per eight columns)
//   [sync 1: the last CTA to arrive sums every column of the partials in a fixed order]
//   Kahan's "twice is enough": the first pass loses more than half of ||w||^2 iff
//   ||h||^2 > ||w||^2 / 2 (Pythagoras, decided before the update).  Otherwise
//   ||w - V h||^2 = ||w||^2 - ||h||^2 within a few units of FP64 rounding (V orthonormal
//   to working accuracy, no cancellation below one half), so the update writes the new
//   column v_{j+1} = (w - V h) / h_{j+1,j} directly: one sync per step.
//   With the second pass: w1 = w - V h; partials of h2 = V^T w1 and ||w1||^2 [sync 2];
//   v_{j+1} = (w1 - V h2) / sqrt(||w1||^2 - ||h2||^2) (h2 is of rounding size).
//   CTA 0 adds h (and h2) to the Hessenberg column and applies the Givens rotations.
// The syncs wait with a bounded spin; an expired wait records DEV_TIMEOUT_GRID and the
// kernel returns.
constexpr int kGmThreads = 512;
constexpr int kGmGroup = 8;   // basis columns per sweep of the partial dot products
template <typename TAZ>
struct GmStepArgs {
  double* V;
  int64_t ld, len, m;
  double* w;
  const TAZ* az;
  GmState* st;
  int maxc, ldh;
  double* Dp;     // [maxc + 1][ldd] partials, one column per block (row ncols: the squared norm)
  double* sq;     // unused (kept for the launch signature)
  double* hsum;   // [maxc + 1] column sums
  double* H;
  double* cs;
  double* sn;
  double* g;
  float* v32;
  unsigned* bar;  // [0]: arrivals, [1]: generation
  int* err;
  int ldd;        // leading dimension of Dp (>= the grid size)
  uint64_t wait_ns;   // limit of each grid-sync wait
  double alpha;       // w_top = alpha v_top + A z (Sec. 4.1 scaling; 1 unscaled)
  unsigned long long* seq;   // MGS: arrival counter of the grid sums (zero before the solve)
  int expire;         // MGS: wait for one arrival more than the grid makes (the timeout test)
};

// Dp[c][block] = sum over rows [r0, r1) of V[c][i] w[i] for c < ncols; Dp[ncols][block] = sum of w[i]^2.
// The (ncols + 1) sums form G groups of eight; the CTA's rows are cut into S slices with
// G x S close to the warp count, and each warp takes one (group, slice) task: its lanes
// stride over the slice two rows at a time (18 loads in flight), one butterfly reduces
// the eight sums over the warp, and one thread per column adds the S slice sums in slice
// order.  Every partial is reduced once, whatever the number of rows per CTA.
constexpr int kGmRed = 160;   // doubles of the slice-sum buffer (>= max(16, G) x 8 with G <= 17)
__device__ __forceinline__ void gm_partials(const double* __restrict__ V, int64_t ld,
                                            const double* __restrict__ w, int64_t r0, int64_t r1,
                                            int ncols, double* Dp, int ldd, double* red /* [kGmRed] */,
                                            int64_t blk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = (ncols + kGmGroup) / kGmGroup;   // groups covering ncols + 1 sums
  const int S = G >= nw ? 1 : nw / G;
  const int64_t per = (r1 - r0 + S - 1) / S;
  for (int task = warp; task < G * S; task += nw) {
    const int g = task % G, sl = task / G, c0 = g * kGmGroup;
    const int64_t s0 = r0 + (int64_t)sl * per, s1 = min(r1, s0 + per);
    double t[kGmGroup];
#pragma unroll
    for (int k = 0; k < kGmGroup; ++k) t[k] = 0.0;
    int64_t i = s0 + lane;
    if (c0 + kGmGroup <= ncols) {   // eight basis columns, no norm
      for (; i + 32 < s1; i += 64) {
        const double wa = w[i], wb = w[i + 32];
        double va[kGmGroup], vb[kGmGroup];
#pragma unroll
        for (int k = 0; k < kGmGroup; ++k) {
          va[k] = V[(int64_t)(c0 + k) * ld + i];
          vb[k] = V[(int64_t)(c0 + k) * ld + i + 32];
        }
#pragma unroll
        for (int k = 0; k < kGmGroup; ++k) t[k] = fma(vb[k], wb, fma(va[k], wa, t[k]));
      }
    }
    for (; i < s1; i += 32) {
      const double wi = w[i];
#pragma unroll
      for (int k = 0; k < kGmGroup; ++k) {
        const int c = c0 + k;
        if (c < ncols) t[k] = fma(V[(int64_t)c * ld + i], wi, t[k]);
        else if (c == ncols) t[k] = fma(wi, wi, t[k]);
      }
    }
    static_assert(kGmGroup == 8, "warp_reduce8 reduces eight sums");
    const double tot = warp_reduce8(t);
    if ((lane & 3) == 0) red[(sl * G + g) * kGmGroup + ((lane >> 2) & 7)] = tot;
  }
  __syncthreads();
  for (int c = threadIdx.x; c <= ncols; c += blockDim.x) {
    const int g = c / kGmGroup, k = c % kGmGroup;
    double s = 0.0;
    for (int sl = 0; sl < S; ++sl) s += red[(sl * G + g) * kGmGroup + k];
    Dp[(int64_t)c * ldd + blk] = s;   // column-major: [column][block]
  }
  __syncthreads();
}

// The last CTA to arrive sums the partials Dp[.][0..cols) (column c by one warp, in
// block order) into hsum and releases the others; every CTA then copies hsum into hs.
// Returns false if the wait ran out.
__device__ __forceinline__ bool gm_sync_sums(double* Dp, int ldd, double* hsum, int cols, unsigned* cnt,
                                             unsigned* gen, int* err, uint64_t wait_ns, double* hs,
                                             int* s_flag) {
  const unsigned nb = gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned ticket = atomicAdd(cnt, 1u);
    s_flag[0] = (ticket == nb - 1) ? 1 : 0;
    s_flag[1] = (int)g;
  }
  __syncthreads();
  int ok = 1;
  if (s_flag[0]) {
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < cols; c += nw) {
      const double* col = Dp + (int64_t)c * ldd;
      double t0 = 0.0, t1 = 0.0;
      unsigned q = lane;
      for (; q + 32 < nb; q += 64) {
        t0 += __ldcg(col + q);
        t1 += __ldcg(col + q + 32);
      }
      if (q < nb) t0 += __ldcg(col + q);
      const double t = warp_sum(t0 + t1);
      if (lane == 0) hsum[c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned* vgen = gen;
    const unsigned g = (unsigned)s_flag[1];
    const uint64_t t0 = globaltimer_ns();
    while (*vgen == g) {
      if (globaltimer_ns() - t0 > wait_ns) {
        set_error(err, DEV_TIMEOUT_GRID);
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  if (__syncthreads_and(ok) == 0) return false;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) hs[c] = __ldcg(hsum + c);
  __syncthreads();
  return true;
}

// w[i] - sum_c V[c][i] h[c] for row i
__device__ __forceinline__ double gm_row_update(const double* __restrict__ V, int64_t ld, double wi,
                                                int64_t i, int ncols, const double* hs) {
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
  int c = 0;
  for (; c + 3 < ncols; c += 4) {
    p0 = fma(V[(int64_t)c * ld + i], hs[c], p0);
    p1 = fma(V[(int64_t)(c + 1) * ld + i], hs[c + 1], p1);
    p2 = fma(V[(int64_t)(c + 2) * ld + i], hs[c + 2], p2);
    p3 = fma(V[(int64_t)(c + 3) * ld + i], hs[c + 3], p3);
  }
  for (; c < ncols; ++c) p0 = fma(V[(int64_t)c * ld + i], hs[c], p0);
  return wi - ((p0 + p1) + (p2 + p3));
}

// The same for rows i and i2 at once (same summation order as gm_row_update): 16 loads
// in flight per thread.
__device__ __forceinline__ void gm_row_update2(const double* __restrict__ V, int64_t ld, int64_t i,
                                               int64_t i2, int ncols, const double* hs, double& wa,
                                               double& wb) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
  int c = 0;
  for (; c + 3 < ncols; c += 4) {
    const double* v0 = V + (int64_t)c * ld;
    const double va0 = v0[i], va1 = v0[ld + i], va2 = v0[2 * ld + i], va3 = v0[3 * ld + i];
    const double vb0 = v0[i2], vb1 = v0[ld + i2], vb2 = v0[2 * ld + i2], vb3 = v0[3 * ld + i2];
    a0 = fma(va0, hs[c], a0);
    a1 = fma(va1, hs[c + 1], a1);
    a2 = fma(va2, hs[c + 2], a2);
    a3 = fma(va3, hs[c + 3], a3);
    b0 = fma(vb0, hs[c], b0);
    b1 = fma(vb1, hs[c + 1], b1);
    b2 = fma(vb2, hs[c + 2], b2);
    b3 = fma(vb3, hs[c + 3], b3);
  }
  for (; c < ncols; ++c) {
    a0 = fma(V[(int64_t)c * ld + i], hs[c], a0);
    b0 = fma(V[(int64_t)c * ld + i2], hs[c], b0);
  }
  wa = wa - ((a0 + a1) + (a2 + a3));
  wb = wb - ((b0 + b1) + (b2 + b3));
}

template <typename TAZ>
__global__ void __launch_bounds__(kGmThreads, 2) gm_step_kernel(const GmStepArgs<TAZ> a) {
  if (a.st->done) return;   // uniform: read before any grid sync
  __shared__ double hs[130];
  __shared__ double red[kGmRed];
  __shared__ double hcol[130];   // block 0: the column j of the Hessenberg matrix
  __shared__ int s_flag[2];
  const int j = a.st->j, ncols = j + 1;
  const int nb = gridDim.x, b = blockIdx.x;
  const int64_t chunk = (a.len + nb - 1) / nb;
  const int64_t r0 = (int64_t)b * chunk, r1 = min(a.len, r0 + chunk);
  const int ldd = a.ldd;
  double* w = a.w;
  const double* V = a.V;
  if (a.az) {   // w_top = alpha v_top + A z (the pass left A z in az); else w_top is formed
    const double* vj = V + (int64_t)j * a.ld;
    const double al = a.alpha;
    for (int64_t i = r0 + threadIdx.x; i < min(r1, a.m); i += blockDim.x) w[i] = fma(al, vj[i], (double)a.az[i]);
    __syncthreads();
  }
  // ---- first pass: h and ||w||^2
  gm_partials(V, a.ld, w, r0, r1, ncols, a.Dp, ldd, red, blockIdx.x);
  if (!gm_sync_sums(a.Dp, ldd, a.hsum, ncols + 1, a.bar, a.bar + 1, a.err, a.wait_ns, hs, s_flag)) {
    if (threadIdx.x == 0) a.st->done = 1;   // later launches of the batch skip; the host reads err
    return;
  }
  const double wn2 = hs[ncols];
  if (threadIdx.x == 0) {   // ||h||^2 in the same order in every CTA
    double q = 0.0;
    for (int c = 0; c < ncols; ++c) q = fma(hs[c], hs[c], q);
    red[0] = q;
  }
  __syncthreads();
  const double hh = red[0];
  __syncthreads();
  const bool second = hh > 0.5 * wn2;
  const int64_t step = blockDim.x;
  if (b == 0) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hcol[c] = hs[c];
    if (threadIdx.x == 0) {
      a.st->reorth = second ? 1 : 0;
      a.st->nreorth += second ? 1 : 0;
    }
  }
  double hn2;
  if (!second) {
    hn2 = wn2 - hh;
  } else {
    int64_t i = r0 + threadIdx.x;
    for (; i + step < r1; i += 2 * step) {
      double wa = w[i], wb = w[i + step];
      gm_row_update2(V, a.ld, i, i + step, ncols, hs, wa, wb);
      w[i] = wa;
      w[i + step] = wb;
    }
    for (; i < r1; i += step) w[i] = gm_row_update(V, a.ld, w[i], i, ncols, hs);
    __syncthreads();   // this CTA's rows of w1 are final for the second pass
    gm_partials(V, a.ld, w, r0, r1, ncols, a.Dp, ldd, red, blockIdx.x);
    if (!gm_sync_sums(a.Dp, ldd, a.hsum, ncols + 1, a.bar, a.bar + 1, a.err, a.wait_ns, hs, s_flag)) {
    if (threadIdx.x == 0) a.st->done = 1;   // later launches of the batch skip; the host reads err
    return;
  }
    if (b == 0)
      for (int c = threadIdx.x; c < ncols; c += blockDim.x) hcol[c] += hs[c];
    if (threadIdx.x == 0) {
      double q = 0.0;
      for (int c = 0; c < ncols; ++c) q = fma(hs[c], hs[c], q);
      red[0] = q;
    }
    __syncthreads();
    hn2 = hs[ncols] - red[0];
    __syncthreads();
  }
  if (!(hn2 > 0.0)) hn2 = 0.0;
  // ---- new column (every block, own rows) and the Givens step (warp 0 of block 0,
  // while the block's other warps take its rows)
  const double inv = hn2 > 0.0 ? 1.0 / sqrt(hn2) : 0.0;
  double* vn = a.V + (int64_t)(j + 1) * a.ld;
  __syncthreads();   // block 0: hcol is complete
  if (b == 0 && threadIdx.x < 32) {
    gm_finish_warp(hn2, a.st, hcol, a.H, a.ldh, a.cs, a.sn, a.g);
    return;
  }
  {
    const int64_t step = (b == 0) ? blockDim.x - 32 : blockDim.x;
    int64_t i = r0 + threadIdx.x - ((b == 0) ? 32 : 0);
    for (; i + step < r1; i += 2 * step) {
      double wa = w[i], wb = w[i + step];
      gm_row_update2(V, a.ld, i, i + step, ncols, hs, wa, wb);
      wa *= inv;
      wb *= inv;
      vn[i] = wa;
      vn[i + step] = wb;
      if (a.v32) {
        if (i < a.m) a.v32[i] = (float)wa;
        if (i + step < a.m) a.v32[i + step] = (float)wb;
      }
    }
    for (; i < r1; i += step) {
      const double v = gm_row_update(V, a.ld, w[i], i, ncols, hs) * inv;
      vn[i] = v;
      if (a.v32 && i < a.m) a.v32[i] = (float)v;
    }
  }
}

// ---------------------------------------------------------------- MGS Arnoldi step
// Modified Gram-Schmidt for long vectors, one cooperative launch per FGMRES iteration.
// Sweep c = 0..j+1 over the CTA's rows: subtract the projection on v_{c-1} (its
// coefficient h_{c-1} is the previous sweep's grid sum) and accumulate v_c^T w (sweep
// j+1: ||w||^2); each sweep ends in one grid sum.  2(j+1) FP64 FMAs per row, the least
// any Gram-Schmidt form needs for j+1 projections (classical Gram-Schmidt with its second
// pass takes 4(j+1)); GB300's FP64 rate, not HBM, bounds the step at m in the millions.
// Each row stays with one thread from sweep to sweep, so w needs no barrier between
// sweeps.  WS: the CTA's rows of w live in shared memory for the whole step (one CTA per
// SM; rows of [r; x] up to 152 x ~27,000), so a sweep reads only v_c from HBM and v_{c-1}
// again (from L2); otherwise w is read and written in global memory every sweep.
constexpr int kMgsThreads = 512;      // global-w form: two CTAs per SM
constexpr int kMgsThreadsWs = 1024;   // shared-w form: one CTA per SM
constexpr int kMgsUnroll = 4;
constexpr int kMgsStaticSmem = 16384; // bound on the kernel's static shared memory

// One grid-wide sum.  Thread 0 of each CTA stores its value in part[b] and takes a
// ticket from a 64-bit arrival counter with a release add; the counter is zeroed before
// the solve and every launch of the solve has the same grid, so the tickets of one sum
// fill [k nb, (k + 1) nb) and the sum is complete when the counter reaches (k + 1) nb.
// Thread 0 waits for that (acquire loads, bounded; plus_one: wait for one more arrival,
// which never comes -- the timeout test), then warp 0 adds the values in block order
// itself, the same order in every CTA, so every CTA gets the same sum.  part is a fresh
// column per sum, so a CTA that has moved on disturbs no one still reading.  *out
// (shared) receives the sum.  Returns false if the wait ran out.
__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool gm_grid_sum_ctr(double* part, unsigned long long* ctr, int plus_one, double mine,
                                                int* err, uint64_t wait_ns, double* out) {
  const unsigned nb = gridDim.x;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
    const unsigned long long ticket = atom_add_release_u64(ctr, 1ull);
    const unsigned long long target = (ticket / nb + 1ull) * nb + (plus_one ? 1ull : 0ull);
    int ok = 1;
    const uint64_t t0 = globaltimer_ns();
    while (ld_acquire_u64(ctr) < target) {
      if (globaltimer_ns() - t0 > wait_ns) {
        set_error(err, DEV_TIMEOUT_GRID);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return false;
  if (threadIdx.x < 32) {
    double t0 = 0.0, t1 = 0.0;
    unsigned q = threadIdx.x;
    for (; q + 32 < nb; q += 64) {
      t0 += __ldcg(part + q);
      t1 += __ldcg(part + q + 32);
    }
    if (q < nb) t0 += __ldcg(part + q);
    const double t = warp_sum(t0 + t1);
    if (threadIdx.x == 0) *out = t;
  }
  __syncthreads();
  return true;
}

template <typename TAZ, bool WS, int NT>
__global__ void __launch_bounds__(NT, WS ? 1 : 2) gm_mgs_kernel(const GmStepArgs<TAZ> a) {
  if (a.st->done) return;   // uniform: read before any grid sync
  extern __shared__ double wsm[];   // WS: w[r0 .. r1)
  __shared__ double hs[130];
  __shared__ double red[NT];
  __shared__ double hcol[130];
  const int j = a.st->j, ncols = j + 1;
  const int nb = gridDim.x, b = blockIdx.x;
  const int64_t chunk = (a.len + nb - 1) / nb;
  const int64_t r0 = (int64_t)b * chunk, r1 = min(a.len, r0 + chunk);
  constexpr int64_t step = NT;
  double* w = WS ? wsm - r0 : a.w;   // indexed by the row
  const double* wg = a.w;
  const double* V = a.V;
  const double* vj = V + (int64_t)j * a.ld;
  const double al = a.alpha;
  const bool form = a.az != nullptr;
  for (int c = 0; c <= ncols; ++c) {
    const double* vp = V + (int64_t)(c > 0 ? c - 1 : 0) * a.ld;
    const double* vc = V + (int64_t)(c < ncols ? c : 0) * a.ld;
    const double hp = c > 0 ? hs[c - 1] : 0.0;
    double t = 0.0;
    int64_t i = r0 + threadIdx.x;
    for (; i + (kMgsUnroll - 1) * step < r1; i += kMgsUnroll * step) {
      double wv[kMgsUnroll], pv[kMgsUnroll], cv[kMgsUnroll];
#pragma unroll
      for (int u = 0; u < kMgsUnroll; ++u) {
        const int64_t q = i + u * step;
        if (c == 0) wv[u] = (form && q < a.m) ? fma(al, vj[q], (double)a.az[q]) : wg[q];
        else wv[u] = w[q];
        pv[u] = c > 0 ? vp[q] : 0.0;
        cv[u] = c < ncols ? vc[q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kMgsUnroll; ++u) {
        const int64_t q = i + u * step;
        if (c > 0) wv[u] = fma(-hp, pv[u], wv[u]);
        if (WS || c > 0 || (form && q < a.m)) w[q] = wv[u];
        t = fma(c < ncols ? cv[u] : wv[u], wv[u], t);
      }
    }
    for (; i < r1; i += step) {
      double wi = c > 0 ? w[i] : ((form && i < a.m) ? fma(al, vj[i], (double)a.az[i]) : wg[i]);
      if (c > 0) wi = fma(-hp, vp[i], wi);
      if (WS || c > 0 || (form && i < a.m)) w[i] = wi;
      t = fma(c < ncols ? vc[i] : wi, wi, t);
    }
    // block sum in a fixed order: NT / 32 values per lane of warp 0 (four interleaved
    // chains), then the warp
    red[threadIdx.x] = t;
    __syncthreads();
    double mine = 0.0;
    if (threadIdx.x < 32) {
      static_assert(NT % 128 == 0, "four chains of NT / 128 values");
      const double* rl = red + threadIdx.x * (NT / 32);
      double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
#pragma unroll
      for (int k = 0; k < NT / 32; k += 4) {
        q0 += rl[k];
        q1 += rl[k + 1];
        q2 += rl[k + 2];
        q3 += rl[k + 3];
      }
      mine = warp_sum((q0 + q1) + (q2 + q3));
    }
    if (!gm_grid_sum_ctr(a.Dp + (int64_t)c * a.ldd, a.seq, a.expire, mine, a.err, a.wait_ns, hs + c)) {
      if (threadIdx.x == 0) a.st->done = 1;   // later launches of the batch skip; the host reads err
      return;
    }
  }
  double hn2 = hs[ncols];
  if (!(hn2 > 0.0)) hn2 = 0.0;
  if (b == 0) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hcol[c] = hs[c];
    if (threadIdx.x == 0) a.st->reorth = 0;
  }
  const double inv = hn2 > 0.0 ? 1.0 / sqrt(hn2) : 0.0;
  double* vn = a.V + (int64_t)(j + 1) * a.ld;
  __syncthreads();   // block 0: hcol is complete; every thread's last w is visible to the CTA
  if (b == 0 && threadIdx.x < 32) {
    gm_finish_warp(hn2, a.st, hcol, a.H, a.ldh, a.cs, a.sn, a.g);
    return;
  }
  const int64_t nstep = (b == 0) ? NT - 32 : NT;
  for (int64_t i = r0 + threadIdx.x - ((b == 0) ? 32 : 0); i < r1; i += nstep) {
    const double v = w[i] * inv;
    vn[i] = v;
    if (a.v32 && i < a.m) a.v32[i] = (float)v;
  }
}

template <typename TAZ>
cudaError_t launch_gm_step(double* V, int64_t ld, double* w, int64_t len, int64_t m, const TAZ* az,
                           GmState* st, int maxc, double* Dp, double* sq, double* hsum, double* H, int ldh,
                           double* cs, double* sn, double* g, float* v32, unsigned* bar, int* err,
                           int num_sms, cudaStream_t s, uint64_t wait_ns, double alpha, int gs,
                           unsigned long long* seq, int expire) {
  static_assert(sizeof(GmStepArgs<TAZ>) < 4096, "kernel parameter block");
  if (maxc > 128 || gs < 0 || gs > 2 || (gs > 0 && seq == nullptr)) return cudaErrorInvalidValue;
  const bool mgs = gs > 0;
  // MGS keeps w in shared memory when one CTA per SM holds its rows (unless gs = 2)
  const int64_t ws_rows = (len + num_sms - 1) / num_sms;
  const size_t ws_bytes = (size_t)ws_rows * 8;
  const bool ws = gs == 1 && ws_bytes + kMgsStaticSmem <= 227 * 1024;
  auto kern = !mgs ? gm_step_kernel<TAZ>
                   : (ws ? gm_mgs_kernel<TAZ, true, kMgsThreadsWs> : gm_mgs_kernel<TAZ, false, kMgsThreads>);
  const int threads = !mgs ? kGmThreads : (ws ? kMgsThreadsWs : kMgsThreads);
  const size_t dyn = ws ? ws_bytes : 0;
  if (ws) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // co-resident CTAs (cooperative launch): two per SM for long vectors (more loads in
  // flight), one per SM otherwise (fewer partials to sum); shared w: one per SM
  const int nblk = ws ? num_sms : num_sms * ((occ >= 2 && len >= ((int64_t)1 << 20)) ? 2 : 1);
  GmStepArgs<TAZ> a{V, ld, len, m, w, az, st, maxc, 0, Dp, sq, hsum, H, cs, sn, g, v32, bar, err};
  a.ldh = ldh;
  a.ldd = 2 * num_sms;   // the caller's Dp holds (maxc + 1) x 2 num_sms values
  a.wait_ns = wait_ns > 0 ? wait_ns : kWaitLimitNs;
  a.alpha = alpha;
  a.seq = seq;
  a.expire = expire;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}
template cudaError_t launch_gm_step<float>(double*, int64_t, double*, int64_t, int64_t, const float*, GmState*,
                                           int, double*, double*, double*, double*, int, double*, double*,
                                           double*, float*, unsigned*, int*, int, cudaStream_t, uint64_t,
                                           double, int, unsigned long long*, int);
template cudaError_t launch_gm_step<double>(double*, int64_t, double*, int64_t, int64_t, const double*,
                                            GmState*, int, double*, double*, double*, double*, int, double*,
                                            double*, double*, float*, unsigned*, int*, int, cudaStream_t,
                                            uint64_t, double, int, unsigned long long*, int);

// y = H[:k,:k]^-1 g[:k]  (k = st->j): one warp, column-oriented back substitution
__global__ void gm_solve_kernel(const GmState* st, const double* H, int ldh, const double* g, double* y) {
  extern __shared__ double hs[];   // k x k, column-major
  __shared__ double rhs[130];
  const int k = st->j, lane = threadIdx.x;
  for (int c = 0; c < k; ++c)
    for (int i = lane; i <= c; i += 32) hs[c * k + i] = H[(int64_t)c * ldh + i];
  for (int i = lane; i < k; i += 32) rhs[i] = g[i];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = rhs[i] / hs[i * k + i];
    __syncwarp();
    for (int l = lane; l < i; l += 32) rhs[l] -= hs[i * k + l] * yi;
    if (lane == 0) y[i] = yi;
    __syncwarp();
  }
}

// d[i] += sum_c B[c][i] y[c] for i < len (B column-major, ld); partial sums of
// the correction squared and of the updated vector squared.
template <typename TB>
__global__ void gm_apply_kernel(const TB* __restrict__ B, int64_t ld, int64_t len, const GmState* st,
                                const double* __restrict__ y, double* __restrict__ d,
                                double* part_dd, double* part_d, double scale) {
  __shared__ double ys[128];
  __shared__ double red[33];
  const int k = st->j;
  for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = y[c];
  __syncthreads();
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    // four interleaved chains, their loads issued together (the loop is latency-bound)
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int c = 0;
    for (; c + 3 < k; c += 4) {
      const TB* bc = B + (int64_t)c * ld + i;
      const double b0 = (double)bc[0], b1 = (double)bc[ld], b2 = (double)bc[2 * ld], b3 = (double)bc[3 * ld];
      a0 = fma(b0, ys[c], a0);
      a1 = fma(b1, ys[c + 1], a1);
      a2 = fma(b2, ys[c + 2], a2);
      a3 = fma(b3, ys[c + 3], a3);
    }
    for (; c < k; ++c) a0 = fma((double)B[(int64_t)c * ld + i], ys[c], a0);
    double acc = ((a0 + a1) + (a2 + a3)) * scale;
    const double nv = d[i] + acc;
    d[i] = nv;
    s1 += acc * acc;
    s2 += nv * nv;
  }
  s1 = block_sum_d(s1, red);
  s2 = block_sum_d(s2, red);
  if (threadIdx.x == 0) {
    part_dd[blockIdx.x] = s1;
    part_d[blockIdx.x] = s2;
  }
}

cudaError_t launch_gm_init(const double* sq_partial, int nblk, GmState* st, double* g, cudaStream_t s) {
  gm_init_kernel<<<1, 256, 0, s>>>(sq_partial, nblk, st, g);
  return cudaGetLastError();
}
cudaError_t launch_gm_solve(const GmState* st, const double* H, int ldh, const double* g, double* y,
                            cudaStream_t s) {
  const size_t smem = (size_t)(ldh - 1) * (ldh - 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dyn_smem(gm_solve_kernel, smem);
    if (e != cudaSuccess) return e;
  }
  gm_solve_kernel<<<1, 32, smem, s>>>(st, H, ldh, g, y);
  return cudaGetLastError();
}
template <typename TB>
cudaError_t launch_gm_apply(const TB* B, int64_t ld, int64_t len, const GmState* st, const double* y,
                            double* d, double* part_dd, double* part_d, int nblk, cudaStream_t s,
                            double scale) {
  gm_apply_kernel<TB><<<nblk, 256, 0, s>>>(B, ld, len, st, y, d, part_dd, part_d, scale);
  return cudaGetLastError();
}
template cudaError_t launch_gm_apply<double>(const double*, int64_t, int64_t, const GmState*, const double*,
                                             double*, double*, double*, int, cudaStream_t, double);
template cudaError_t launch_gm_apply<float>(const float*, int64_t, int64_t, const GmState*, const double*,
                                            double*, double*, double*, int, cudaStream_t, double);

cudaError_t launch_sum_partials(const double* partial, int nblk, double* out, bool take_sqrt,
                                cudaStream_t st) {
  sum_partials_kernel<<<1, 1024, 0, st>>>(partial, nblk, out, take_sqrt);
  return cudaGetLastError();
}

// Copies [f; h] into V[:, 0] and leaves partial sums of squares.
__global__ void gm_rhs_kernel(const double* __restrict__ f, const double* __restrict__ h, int64_t m,
                              int64_t n, double* __restrict__ V0, double* sq_partial, double alpha) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m + n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (i < m) ? f[i] : (alpha == 1.0 ? h[i - m] : h[i - m] / alpha);
    V0[i] = v;
    s += v * v;
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) sq_partial[blockIdx.x] = s;
}

cudaError_t launch_gm_rhs(const double* f, const double* h, int64_t m, int64_t n, double* V0,
                          double* sq_partial, int nblk, cudaStream_t s, double alpha) {
  gm_rhs_kernel<<<nblk, 256, 0, s>>>(f, h, m, n, V0, sq_partial, alpha);
  return cudaGetLastError();
}

// V[:, 0] *= inv_h (after gm_init)
__global__ void gm_scale0_kernel(double* V0, int64_t len, const GmState* st, float* v32, int64_t m) {
  const double s = st->inv_h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = V0[i] * s;
    V0[i] = v;
    if (v32 && i < m) v32[i] = (float)v;
  }
}
cudaError_t launch_gm_scale0(double* V0, int64_t len, const GmState* st, float* v32, int64_t m,
                             int nblk, cudaStream_t s) {
  gm_scale0_kernel<<<nblk, 256, 0, s>>>(V0, len, st, v32, m);
  return cudaGetLastError();
}


// ============================================================ grouped (batched) forms
// Problem p owns CTAs [start[p], start[p + 1]) of each launch; its block index and
// block count within the launch stand in for blockIdx.x and gridDim.x of the
// single-problem kernels above, whose bodies these call.

// Persistent over the items (problem, block of the problem's pass): CTA b takes items b,
// b + gridDim.x, ...; every item is computed exactly as a CTA of that problem's own pass
// would compute it, so the result does not depend on the grid size.
template <typename T, int VW, int VPL, int MODE>
__global__ void __launch_bounds__(256)
    grouped_pass_kernel(const PassArgs<T>* __restrict__ tab, const int* __restrict__ start, int nprob,
                        int64_t items) {
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int pr = group_of(start, nprob, it);
    pass_body<T, VW, VPL, MODE>(tab[pr], it - start[pr], (int64_t)start[pr + 1] - start[pr]);
    __syncthreads();   // the item's shared-memory reduction is read before the next item writes it
  }
}

template <typename T>
cudaError_t launch_grouped_pass(int mode, int vw, int vpl, const PassArgs<T>* tab, const int* start,
                                int64_t ctas, int nprob, size_t smem, cudaStream_t st, int64_t grid) {
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 2147483647LL) return cudaErrorInvalidValue;
  const int64_t g = (grid > 0 && grid < ctas) ? grid : ctas;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)g, 256, smem, st>>>(tab, start, nprob, ctas);
    return cudaGetLastError();
  };
  if constexpr (sizeof(T) == 4) {
    if (vw != 4 || vpl != 2) return cudaErrorInvalidValue;
    if (mode == PM_LSQR) return go(grouped_pass_kernel<float, 4, 2, PM_LSQR>);
    if (mode == PM_FGM) return go(grouped_pass_kernel<float, 4, 2, PM_FGM>);
  } else {
    if (vw != 1 || vpl != 8) return cudaErrorInvalidValue;
    if (mode == PM_LSQR) return go(grouped_pass_kernel<double, 1, 8, PM_LSQR>);
    if (mode == PM_FGM) return go(grouped_pass_kernel<double, 1, 8, PM_FGM>);
    if (mode == PM_RES) return go(grouped_pass_kernel<double, 1, 8, PM_RES>);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_grouped_pass<float>(int, int, int, const PassArgs<float>*, const int*, int64_t, int,
                                                size_t, cudaStream_t, int64_t);
template cudaError_t launch_grouped_pass<double>(int, int, int, const PassArgs<double>*, const int*, int64_t, int,
                                                 size_t, cudaStream_t, int64_t);

template <typename TP, typename TO>
__global__ void grouped_colsum_kernel(const GColsum<TP, TO>* __restrict__ tab, const int* __restrict__ start,
                                      int nprob) {
  const int pr = group_of(start, nprob, blockIdx.x);
  const GColsum<TP, TO>& g = tab[pr];
  colsum_body<TP, TO>(g.P, g.nblk, g.n, g.scale_ptr, g.scale_mul, g.out, g.done, (int64_t)blockIdx.x - start[pr]);
}

template <typename TP, typename TO>
cudaError_t launch_grouped_colsum(const GColsum<TP, TO>* tab, const int* start, int64_t ctas, int nprob,
                                  cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  grouped_colsum_kernel<TP, TO><<<(unsigned)ctas, dim3(32, 32), 0, st>>>(tab, start, nprob);
  return cudaGetLastError();
}
template cudaError_t launch_grouped_colsum<float, float>(const GColsum<float, float>*, const int*, int64_t, int,
                                                         cudaStream_t);
template cudaError_t launch_grouped_colsum<double, double>(const GColsum<double, double>*, const int*, int64_t,
                                                           int, cudaStream_t);

template <typename TP>
__global__ void grouped_lsqr_colsum_kernel(const GLsqrColsum<TP>* __restrict__ tab, const int* __restrict__ start,
                                           int nprob, bool init) {
  const int pr = group_of(start, nprob, blockIdx.x);
  const GLsqrColsum<TP>& g = tab[pr];
  lsqr_colsum_body<TP>(g.P, g.nblk, g.n, g.sq, g.st, init, g.out, (int64_t)blockIdx.x - start[pr]);
}

template <typename TP>
cudaError_t launch_grouped_lsqr_colsum(const GLsqrColsum<TP>* tab, const int* start, int64_t ctas, int nprob,
                                       bool init, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  grouped_lsqr_colsum_kernel<TP><<<(unsigned)ctas, dim3(32, 32), 0, st>>>(tab, start, nprob, init);
  return cudaGetLastError();
}
template cudaError_t launch_grouped_lsqr_colsum<float>(const GLsqrColsum<float>*, const int*, int64_t, int, bool,
                                                       cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(kTrsvThreads)
    grouped_lsqr_step_kernel(const GLsqrStep<T>* __restrict__ tab, bool init) {
  const GLsqrStep<T>& g = tab[blockIdx.x];
  lsqr_step_body<T>(g.f, g.s, g.v, g.w, g.z, g.t, g.st, init);
}

template <typename T>
cudaError_t launch_grouped_lsqr_step(const GLsqrStep<T>* tab, int nprob, bool init, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  const size_t smem = TrsvSmem<T>::bytes;
  cudaError_t e = allow_dyn_smem(grouped_lsqr_step_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  grouped_lsqr_step_kernel<T><<<(unsigned)nprob, kTrsvThreads, smem, st>>>(tab, init);
  return cudaGetLastError();
}
template cudaError_t launch_grouped_lsqr_step<float>(const GLsqrStep<float>*, int, bool, cudaStream_t);

template <typename TX, typename TY, typename TO>
__global__ void grouped_axpby_kernel(const GAxpby<TX, TY, TO>* __restrict__ tab, const int* __restrict__ start,
                                     int nprob) {
  const int pr = group_of(start, nprob, blockIdx.x);
  const GAxpby<TX, TY, TO>& g = tab[pr];
  if (g.done && *g.done) return;
  const int64_t i = ((int64_t)blockIdx.x - start[pr]) * blockDim.x + threadIdx.x;
  if (i >= g.len) return;
  double v = (double)g.x[i] * g.a;
  if (g.y) v += (double)g.y[i] * g.b;
  g.out[i] = (TO)v;
}

template <typename TX, typename TY, typename TO>
cudaError_t launch_grouped_axpby(const GAxpby<TX, TY, TO>* tab, const int* start, int64_t ctas, int nprob,
                                 cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  grouped_axpby_kernel<TX, TY, TO><<<(unsigned)ctas, 256, 0, st>>>(tab, start, nprob);
  return cudaGetLastError();
}
template cudaError_t launch_grouped_axpby<double, double, float>(const GAxpby<double, double, float>*, const int*,
                                                                 int64_t, int, cudaStream_t);
template cudaError_t launch_grouped_axpby<float, double, double>(const GAxpby<float, double, double>*, const int*,
                                                                 int64_t, int, cudaStream_t);
template cudaError_t launch_grouped_axpby<double, double, double>(const GAxpby<double, double, double>*,
                                                                  const int*, int64_t, int, cudaStream_t);

// ||x|| by one CTA per problem
__global__ void grouped_norm_kernel(const GNorm* __restrict__ tab) {
  __shared__ double red[33];
  const GNorm& g = tab[blockIdx.x];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < g.len; i += blockDim.x) s += g.x[i] * g.x[i];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) *g.out = sqrt(s);
}

cudaError_t launch_grouped_norm(const GNorm* tab, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  grouped_norm_kernel<<<(unsigned)nprob, 1024, 0, st>>>(tab);
  return cudaGetLastError();
}

// ---- FGMRES
// rhs: V[:, 0] = [f; h / alpha] over the problem's CTAs, partial sums of squares
__global__ void grouped_gm_rhs_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob) {
  __shared__ double red[33];
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  double s = 0.0;
  if (!*g.skip) {
    for (int64_t i = blk * blockDim.x + threadIdx.x; i < g.m + g.n; i += nb * blockDim.x) {
      const double v = (i < g.m) ? g.f[i] : (g.alpha == 1.0 ? g.h[i - g.m] : g.h[i - g.m] / g.alpha);
      g.V[i] = v;
      s += v * v;
    }
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) g.sqp[blk] = s;
}

// beta = ||[f; h / alpha]|| (partials in CTA order), state reset, g = beta e_1
__global__ void grouped_gm_init_kernel(const GGm* __restrict__ tab, const int* __restrict__ start) {
  __shared__ double red[33];
  const GGm& g = tab[blockIdx.x];
  const int nb = start[blockIdx.x + 1] - start[blockIdx.x];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += g.sqp[b];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    GmState* st = g.st;
    const double beta = sqrt(s);
    st->beta0 = beta;
    st->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
    st->j = 0;
    st->relres = beta > 0.0 ? 1.0 : 0.0;
    st->reorth = 0;
    st->nreorth = 0;
    st->done = (*g.skip || beta == 0.0 || st->maxit <= 0) ? 1 : 0;
    g.g[0] = beta;
  }
}

__global__ void grouped_gm_scale0_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob) {
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  if (g.st->done) return;
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  const double sc = g.st->inv_h;
  for (int64_t i = blk * blockDim.x + threadIdx.x; i < g.m + g.n; i += nb * blockDim.x) {
    const double v = g.V[i] * sc;
    g.V[i] = v;
    if (g.v32 && i < g.m) g.v32[i] = (float)v;
  }
}

cudaError_t launch_grouped_gm_init(const GGm* tab, const int* start, int64_t ctas, int nprob, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  grouped_gm_rhs_kernel<<<(unsigned)ctas, 256, 0, st>>>(tab, start, nprob);
  grouped_gm_init_kernel<<<(unsigned)nprob, 256, 0, st>>>(tab, start);
  grouped_gm_scale0_kernel<<<(unsigned)ctas, 256, 0, st>>>(tab, start, nprob);
  return cudaGetLastError();
}

// Arnoldi, phase A (second = 0): w_top = alpha v_top + A z (unless the pass formed it), then
// the partials of V^T w and ||w||^2 over the CTA's rows; phase A' (second = 1, problems
// whose first pass lost more than half of ||w||^2): the same partials of w1.
__global__ void __launch_bounds__(kGmThreads)
    garn_partials_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob, int second) {
  __shared__ double red[kGmRed];
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  const GmState* st = g.st;
  if (st->done || (second && !st->reorth)) return;
  const int j = st->j, ncols = j + 1;
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  const int64_t len = g.m + g.n, chunk = (len + nb - 1) / nb;
  const int64_t r0 = blk * chunk, r1 = min(len, r0 + chunk);
  if (!second && g.az) {
    const double* vj = g.V + (int64_t)j * g.ld;
    const double al = g.alpha;
    for (int64_t i = r0 + threadIdx.x; i < min(r1, g.m); i += blockDim.x) {
      const double azi = g.az_f32 ? (double)static_cast<const float*>(g.az)[i] : static_cast<const double*>(g.az)[i];
      g.w[i] = fma(al, vj[i], azi);
    }
    __syncthreads();
  }
  gm_partials(g.V, g.ld, g.w, r0, r1, ncols, g.Dp, (int)nb, red, blk);
}

// phase B / B' (one CTA per problem): column sums of the partials in block order, then the
// twice-is-enough test (first pass) and the squared norm of the new column
__global__ void __launch_bounds__(kGmThreads)
    garn_reduce_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int second) {
  const GGm& g = tab[blockIdx.x];
  GmState* st = g.st;
  if (st->done || (second && !st->reorth)) return;
  const int j = st->j, ncols = j + 1;
  const int nb = start[blockIdx.x + 1] - start[blockIdx.x];
  double* hs = second ? g.hs2 : g.hs1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c <= ncols; c += nw) {
    const double* col = g.Dp + (int64_t)c * nb;
    double t0 = 0.0, t1 = 0.0;
    int q = lane;
    for (; q + 32 < nb; q += 64) {
      t0 += col[q];
      t1 += col[q + 32];
    }
    if (q < nb) t0 += col[q];
    const double tt = warp_sum(t0 + t1);
    if (lane == 0) hs[c] = tt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int c = 0; c < ncols; ++c) q = fma(hs[c], hs[c], q);
    const double wn2 = hs[ncols];
    if (!second) {
      const int re = q > 0.5 * wn2 ? 1 : 0;
      st->reorth = re;
      st->nreorth += re;
      const double hn2 = wn2 - q;
      g.hs1[ncols + 1] = hn2 > 0.0 ? hn2 : 0.0;   // used when there is no second pass
    } else {
      const double hn2 = wn2 - q;
      g.hs2[ncols + 1] = hn2 > 0.0 ? hn2 : 0.0;
    }
  }
}

// phase C1 (second pass problems): w1 = w - V h over the CTA's rows
__global__ void __launch_bounds__(kGmThreads)
    garn_sub_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob) {
  __shared__ double hs[130];
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  const GmState* st = g.st;
  if (st->done || !st->reorth) return;
  const int j = st->j, ncols = j + 1;
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  const int64_t len = g.m + g.n, chunk = (len + nb - 1) / nb;
  const int64_t r0 = blk * chunk, r1 = min(len, r0 + chunk);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = g.hs1[c];
  __syncthreads();
  const int64_t step = blockDim.x;
  int64_t i = r0 + threadIdx.x;
  for (; i + step < r1; i += 2 * step) {
    double wa = g.w[i], wb = g.w[i + step];
    gm_row_update2(g.V, g.ld, i, i + step, ncols, hs, wa, wb);
    g.w[i] = wa;
    g.w[i + step] = wb;
  }
  for (; i < r1; i += step) g.w[i] = gm_row_update(g.V, g.ld, g.w[i], i, ncols, hs);
}

// phase C: v_{j+1} = (w - V h) / ||w - V h|| over the CTA's rows (h of the last pass)
__global__ void __launch_bounds__(kGmThreads)
    garn_newcol_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob) {
  __shared__ double hs[130];
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  const GmState* st = g.st;
  if (st->done) return;
  const int j = st->j, ncols = j + 1;
  const double* hsrc = st->reorth ? g.hs2 : g.hs1;
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  const int64_t len = g.m + g.n, chunk = (len + nb - 1) / nb;
  const int64_t r0 = blk * chunk, r1 = min(len, r0 + chunk);
  for (int c = threadIdx.x; c <= ncols; c += blockDim.x) hs[c] = hsrc[c == ncols ? ncols + 1 : c];
  __syncthreads();
  const double hn2 = hs[ncols];
  const double inv = hn2 > 0.0 ? 1.0 / sqrt(hn2) : 0.0;
  double* vn = g.V + (int64_t)(j + 1) * g.ld;
  const int64_t step = blockDim.x;
  int64_t i = r0 + threadIdx.x;
  for (; i + step < r1; i += 2 * step) {
    double wa = g.w[i], wb = g.w[i + step];
    gm_row_update2(g.V, g.ld, i, i + step, ncols, hs, wa, wb);
    wa *= inv;
    wb *= inv;
    vn[i] = wa;
    vn[i + step] = wb;
    if (g.v32) {
      if (i < g.m) g.v32[i] = (float)wa;
      if (i + step < g.m) g.v32[i + step] = (float)wb;
    }
  }
  for (; i < r1; i += step) {
    const double v = gm_row_update(g.V, g.ld, g.w[i], i, ncols, hs) * inv;
    vn[i] = v;
    if (g.v32 && i < g.m) g.v32[i] = (float)v;
  }
}

// phase D (one warp per problem): Hessenberg column h (+ h2), Givens step, j + 1
__global__ void garn_finish_kernel(const GGm* __restrict__ tab) {
  __shared__ double hcol[130];
  const GGm& g = tab[blockIdx.x];
  GmState* st = g.st;
  if (st->done) return;
  const int j = st->j, ncols = j + 1;
  const int re = st->reorth;
  for (int c = threadIdx.x; c < ncols; c += 32) hcol[c] = re ? g.hs1[c] + g.hs2[c] : g.hs1[c];
  __syncwarp();
  const double hn2 = re ? g.hs2[ncols + 1] : g.hs1[ncols + 1];
  gm_finish_warp(hn2, st, hcol, g.H, g.ldh, g.cs, g.sn, g.g);
}

cudaError_t launch_grouped_arnoldi(const GGm* tab, const int* start, int64_t ctas, int nprob, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  const unsigned nc = (unsigned)ctas, np = (unsigned)nprob;
  garn_partials_kernel<<<nc, kGmThreads, 0, st>>>(tab, start, nprob, 0);
  garn_reduce_kernel<<<np, kGmThreads, 0, st>>>(tab, start, 0);
  garn_sub_kernel<<<nc, kGmThreads, 0, st>>>(tab, start, nprob);
  garn_partials_kernel<<<nc, kGmThreads, 0, st>>>(tab, start, nprob, 1);
  garn_reduce_kernel<<<np, kGmThreads, 0, st>>>(tab, start, 1);
  garn_newcol_kernel<<<nc, kGmThreads, 0, st>>>(tab, start, nprob);
  garn_finish_kernel<<<np, 32, 0, st>>>(tab);
  return cudaGetLastError();
}

// update: y = H^-1 g (one warp per problem), then r += alpha V_top y, x += Z y over the
// problem's CTAs with the partial sums of ||alpha V_top y||^2, ||r||^2, ||Z y||^2, ||x||^2
__global__ void grouped_gm_solve_kernel(const GGm* __restrict__ tab) {
  extern __shared__ double hsm[];   // k x k, column-major
  __shared__ double rhs[130];
  const GGm& g = tab[blockIdx.x];
  if (*g.skip) return;
  const int k = g.st->j, lane = threadIdx.x;
  for (int c = 0; c < k; ++c)
    for (int i = lane; i <= c; i += 32) hsm[c * k + i] = g.H[(int64_t)c * g.ldh + i];
  for (int i = lane; i < k; i += 32) rhs[i] = g.g[i];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = rhs[i] / hsm[i * k + i];
    __syncwarp();
    for (int l = lane; l < i; l += 32) rhs[l] -= hsm[i * k + l] * yi;
    if (lane == 0) g.y[i] = yi;
    __syncwarp();
  }
}

__global__ void grouped_gm_apply_kernel(const GGm* __restrict__ tab, const int* __restrict__ start, int nprob) {
  __shared__ double ys[128];
  __shared__ double red[33];
  const int pr = group_of(start, nprob, blockIdx.x);
  const GGm& g = tab[pr];
  const int64_t blk = (int64_t)blockIdx.x - start[pr], nb = (int64_t)start[pr + 1] - start[pr];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (!*g.skip) {
    const int k = g.st->j;
    for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = g.y[c];
    __syncthreads();
    for (int64_t i = blk * blockDim.x + threadIdx.x; i < g.m; i += nb * blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < k; ++c) acc += g.V[(int64_t)c * g.ld + i] * ys[c];
      acc *= g.alpha;
      const double nv = g.r[i] + acc;
      g.r[i] = nv;
      s[0] += acc * acc;
      s[1] += nv * nv;
    }
    for (int64_t i = blk * blockDim.x + threadIdx.x; i < g.n; i += nb * blockDim.x) {
      double acc = 0.0;
      if (g.zb_f32)
        for (int c = 0; c < k; ++c) acc += (double)static_cast<const float*>(g.Zb)[(int64_t)c * g.ldz + i] * ys[c];
      else
        for (int c = 0; c < k; ++c) acc += static_cast<const double*>(g.Zb)[(int64_t)c * g.ldz + i] * ys[c];
      const double nv = g.x[i] + acc;
      g.x[i] = nv;
      s[2] += acc * acc;
      s[3] += nv * nv;
    }
  }
  for (int q = 0; q < 4; ++q) {
    const double v = block_sum_d(s[q], red);
    if (threadIdx.x == 0) g.p4[q * nb + blk] = v;
  }
}

__global__ void grouped_gm_norms_kernel(const GGm* __restrict__ tab, const int* __restrict__ start) {
  __shared__ double red[33];
  const GGm& g = tab[blockIdx.x];
  const int nb = start[blockIdx.x + 1] - start[blockIdx.x];
  for (int q = 0; q < 4; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += g.p4[q * nb + b];
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) g.nrm[q] = s;
  }
}

cudaError_t launch_grouped_gm_update(const GGm* tab, const int* start, int64_t ctas, int nprob,
                                     cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  const size_t smem = (size_t)kMaxGmresBatch * kMaxGmresBatch * 8;
  cudaError_t e = allow_dyn_smem(grouped_gm_solve_kernel, smem);
  if (e != cudaSuccess) return e;
  grouped_gm_solve_kernel<<<(unsigned)nprob, 32, smem, st>>>(tab);
  grouped_gm_apply_kernel<<<(unsigned)ctas, 256, 0, st>>>(tab, start, nprob);
  grouped_gm_norms_kernel<<<(unsigned)nprob, 256, 0, st>>>(tab, start);
  return cudaGetLastError();
}

}  // namespace lsq
