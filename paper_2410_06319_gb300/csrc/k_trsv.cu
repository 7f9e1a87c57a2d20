// Triangular solves with the sketched R (Alg. 2: x_s = R^-1 c, the right
// preconditioner R^-1 in LSQR and FGMRES, the left preconditioner R^-T, and
// h = R^-T g in u_r).
//
// One CTA of 1024 threads, the right-hand side in shared memory, blocks of 32
// rows.  The inverses of the 32 x 32 diagonal blocks are formed once per R
// (dinv_kernel), so a block step is a 32 x 32 matrix-vector product by warp 0
// followed by a rank-32 update of the remaining rows by all threads; there is
// no serial substitution chain inside a block.  The matrices are R (upper) and
// L = R^T (lower), both column-major, so every update reads contiguous column
// segments, which cp.async stages into shared memory ahead of the step that
// uses them (trsv.cuh).
#include <algorithm>

#include "common.cuh"
#include "batch.h"
#include "kernels.h"
#include "trsv.cuh"

namespace lsq {

template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_kernel(const T* __restrict__ M, int64_t ld, const T* __restrict__ D, int n,
                const TIN* __restrict__ y, double yscale, TOUT* __restrict__ x, const int* done,
                const int* jp, int64_t ys, int64_t xstr, int* err) {
  if (done && *done) return;
  if (jp) {  // column j of a basis: offsets read on the device (graph-replayable)
    const int64_t j = *jp;
    y += j * ys;
    x += j * xstr;
  }
  __shared__ T xs[1024];
  extern __shared__ __align__(16) unsigned char trsv_buf[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (T)((double)y[i] * yscale);
  __syncthreads();
  if (!block_trsv<T, UPPER>(M, ld, D, n, xs, trsv_buf, err)) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = (TOUT)xs[i];
}

// ------------------------------------------------------------ cluster solve
// One thread-block cluster of kTrsvCl CTAs (256 threads each).  Block row k (32
// rows) belongs to CTA k % kTrsvCl; its warp (k / kTrsvCl) holds the block's
// right-hand side in registers and the block's row panel of the matrix in shared
// memory for the whole solve (row panels are contiguous in the transposed copy:
// R's rows are L's columns and vice versa).  Steps run as a data flow: when
// x_j arrives (an st.async of 32 values into every CTA's shared memory, which
// completes that CTA's mbarrier j), each owner warp of a pending block applies
// y_k -= M_kj x_j; once its last dependency is in, it forms x_k = D_k^-1 y_k and
// sends it.  The critical path per block is one shared-memory hop across the
// cluster plus two 32 x 32 products.
constexpr int kTrsvCl = 8;
constexpr int kTrsvClThreads = 256;

// 16 bytes into another CTA's shared memory, completing `rbar` there by 16 bytes.
__device__ __forceinline__ void st_async_16(uint32_t raddr, uint4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   raddr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar)
               : "memory");
}
template <typename T>
__device__ __forceinline__ void st_async_remote(uint32_t raddr, T v, uint32_t rbar) {
  if constexpr (sizeof(T) == 4)
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr),
                 "r"(__float_as_uint(v)), "r"(rbar)
                 : "memory");
  else
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
                 "l"(__double_as_longlong(v)), "r"(rbar)
                 : "memory");
}
// Bounded wait on a local mbarrier completed by remote st.async (cluster-scope
// acquire).  Polls with the non-blocking test_wait: the solve's critical path is
// one such wait per block, and a suspended try_wait wakes late.
__device__ __forceinline__ bool cl_wait(uint32_t bar, int* err) {
  auto try_once = [&]() {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    return ok != 0;
  };
  if (try_once()) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!try_once()) {
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      set_error(err, DEV_TIMEOUT_FULL);
      return false;
    }
  }
  return true;
}

// Panel geometry of block row k: width in columns (multiple of 32), row stride
// in elements (16-byte multiple whose 16-byte count is odd: conflict-free
// 16-byte reads of 8 consecutive rows), bytes.
template <typename T>
struct ClPanel {
  static constexpr int VE = 16 / (int)sizeof(T);
  __host__ __device__ static int width(bool upper, int k, int nb) { return upper ? 32 * (nb - 1 - k) : 32 * k; }
  __host__ __device__ static int stride(int w) { return w + VE; }
  __host__ __device__ static size_t bytes(int w) { return w ? (size_t)32 * stride(w) * sizeof(T) : 0; }
};

// Shared memory of CTA `q`: its panels, its diagonal inverses, x of every block, nb mbarriers.
template <typename T>
__host__ __device__ inline size_t cl_smem(bool upper, int n, int q) {
  const int nb = (n + 31) / 32;
  size_t b = 0;
  for (int k = q; k < nb; k += kTrsvCl) b += ClPanel<T>::bytes(ClPanel<T>::width(upper, k, nb)) + 1024 * sizeof(T);
  return b + (((size_t)32 * nb * sizeof(T) + 8 * (size_t)nb + 15) & ~(size_t)15);
}

template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvClThreads)
    trsv_cluster_kernel(const T* __restrict__ Q, int64_t ld, const T* __restrict__ D, int n,
                        const TIN* __restrict__ y, double yscale, TOUT* __restrict__ x, const int* done,
                        const int* jp, int64_t ys, int64_t xstr, int* err) {
  using P = ClPanel<T>;
  if (done && *done) return;   // uniform over the cluster: no CTA reaches a cluster barrier
  if (jp) {
    const int64_t j = *jp;
    y += j * ys;
    x += j * xstr;
  }
  extern __shared__ __align__(16) unsigned char cl_buf[];
  const int nb = (n + 31) >> 5;
  const uint32_t q = cl_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- layout: [x: 32 nb][bars: nb][panels of owned blocks][D of owned blocks]; x and
  // the barriers sit at the same offsets in every CTA (remote addresses are mapped)
  T* xall = reinterpret_cast<T*>(cl_buf);
  uint64_t* bars = reinterpret_cast<uint64_t*>(cl_buf + (size_t)32 * nb * sizeof(T));
  unsigned char* cur = cl_buf + (((size_t)32 * nb * sizeof(T) + 8 * (size_t)nb + 15) & ~(size_t)15);
  T* panel[kTrsvClThreads / 32];
  T* dblk[kTrsvClThreads / 32];
  int nown = 0;
  for (int k = (int)q; k < nb; k += kTrsvCl) {
    panel[nown] = reinterpret_cast<T*>(cur);
    cur += P::bytes(P::width(UPPER, k, nb));
    ++nown;
  }
  for (int t = 0; t < nown; ++t) {
    dblk[t] = reinterpret_cast<T*>(cur);
    cur += 1024 * sizeof(T);
  }
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t xall0 = smem_u32(xall);
  __shared__ uint64_t load_bar;
  const uint32_t lbar = smem_u32(&load_bar);
  // ---- barriers: one per block (its x arrives as 32 * sizeof(T) bytes), one for the loads
  if (tid == 0) {
    for (int k = 0; k < nb; ++k) mbar_init(bar0 + 8 * k, 1);
    mbar_init(lbar, 1);
    fence_barrier_init();
    for (int k = 0; k < nb; ++k) mbar_arrive_expect_tx(bar0 + 8 * k, 32u * (uint32_t)sizeof(T));
  }
  // zero what the copies do not cover: the column tail past the matrix (the
  // partial last column block) and the rows past the matrix (the partial last block)
  for (int t = 0; t < nown; ++t) {
    const int k = (int)q + t * kTrsvCl;
    const int w = P::width(UPPER, k, nb);
    if (!w) continue;
    const int c0 = UPPER ? 32 * (k + 1) : 0;                 // first column of the panel
    const int valid = min(w, n - c0);                        // columns inside the matrix
    const int copied = (valid + P::VE - 1) / P::VE * P::VE;
    const int rows = min(32, n - 32 * k);
    const int tail = w - copied;
    for (int e = tid; e < rows * tail; e += blockDim.x)
      panel[t][(e / tail) * P::stride(w) + copied + e % tail] = T(0);
    for (int e = tid; e < (32 - rows) * w; e += blockDim.x)
      panel[t][(rows + e / w) * P::stride(w) + e % w] = T(0);
  }
  fence_proxy_async_smem();
  __syncthreads();
  // ---- bulk loads: panel rows (contiguous in Q), diagonal inverses
  if (warp == 0) {
    uint32_t bytes = 0;
    for (int t = 0; t < nown; ++t) {
      const int k = (int)q + t * kTrsvCl;
      const int w = P::width(UPPER, k, nb);
      const int c0 = UPPER ? 32 * (k + 1) : 0;
      const int valid = w ? min(w, n - c0) : 0;
      const uint32_t seg = (uint32_t)((valid + P::VE - 1) / P::VE * 16);
      const int rows = min(32, n - 32 * k);
      bytes += 1024u * (uint32_t)sizeof(T) + (seg ? seg * (uint32_t)rows : 0u);
    }
    if (lane == 0) mbar_arrive_expect_tx(lbar, bytes);
    __syncwarp();
    for (int t = 0; t < nown; ++t) {
      const int k = (int)q + t * kTrsvCl;
      const int w = P::width(UPPER, k, nb);
      const int c0 = UPPER ? 32 * (k + 1) : 0;
      const int valid = w ? min(w, n - c0) : 0;
      const uint32_t seg = (uint32_t)((valid + P::VE - 1) / P::VE * 16);
      const int rows = min(32, n - 32 * k);
      if (lane == 0) bulk_load(smem_u32(dblk[t]), D + (size_t)k * 1024, 1024u * (uint32_t)sizeof(T), lbar);
      if (seg && lane < rows)
        bulk_load(smem_u32(panel[t] + lane * P::stride(w)), Q + (size_t)(32 * k + lane) * ld + c0, seg, lbar);
    }
  }
  // every CTA's barriers are initialised before anyone sends
  cl_sync();
  // ---- block warps
  if (warp < nown) {
    const int t = warp;
    const int k = (int)q + t * kTrsvCl;
    const int w = P::width(UPPER, k, nb);
    const int rows = min(32, n - 32 * k);
    T acc = (lane < rows) ? (T)((double)y[32 * k + lane] * yscale) : T(0);
    bool ok = mbar_wait(lbar, 0, err, DEV_TIMEOUT_FULL);
    const T* pr = panel[t] + lane * P::stride(w);
    // dependencies: UPPER j = nb-1 .. k+1, LOWER j = 0 .. k-1 (the order they are produced)
    const int ndep = UPPER ? nb - 1 - k : k;
    for (int d = 0; d < ndep && ok; ++d) {
      const int j = UPPER ? nb - 1 - d : d;
      ok = cl_wait(bar0 + 8 * j, err);
      if (!ok) break;
      const int off = UPPER ? 32 * (j - k - 1) : 32 * j;
      const T* xj = xall + 32 * j;
      T s = T(0);
#pragma unroll
      for (int c = 0; c < 32; c += P::VE) {
        if constexpr (sizeof(T) == 4) {
          const float4 mv = *reinterpret_cast<const float4*>(pr + off + c);
          const float4 xv = *reinterpret_cast<const float4*>(xj + c);
          s += mv.x * xv.x + mv.y * xv.y + mv.z * xv.z + mv.w * xv.w;
        } else {
          const double2 mv = *reinterpret_cast<const double2*>(pr + off + c);
          const double2 xv = *reinterpret_cast<const double2*>(xj + c);
          s += mv.x * xv.x + mv.y * xv.y;
        }
      }
      acc -= s;
    }
    // x_k = D_k^-1 y_k (lane r: sum_c D[c][r] y_c), then to every CTA of the cluster
    const T* dk = dblk[t];
    T xa = T(0), xb = T(0);
#pragma unroll 8
    for (int c = 0; c < 32; c += 2) {
      xa += dk[c * 32 + lane] * __shfl_sync(0xffffffffu, acc, c);
      xb += dk[(c + 1) * 32 + lane] * __shfl_sync(0xffffffffu, acc, c + 1);
    }
    T xk = xa + xb;
    if (lane >= rows) xk = T(0);
    // send x_k: 16-byte pieces, destinations spread over the lanes (lane l serves
    // CTA l % 8, pieces l / 8, l / 8 + 4, ...)
    constexpr int EP = 16 / (int)sizeof(T);                 // elements per piece
    constexpr int PIECES = 32 / EP;                         // pieces per destination
    const uint32_t dst = (uint32_t)(lane & (kTrsvCl - 1));
    const uint32_t rx = cl_map(xall0 + (uint32_t)(32 * k * sizeof(T)), dst);
    const uint32_t rb = cl_map(bar0 + 8 * k, dst);
#pragma unroll
    for (int pc = lane / kTrsvCl; pc < PIECES; pc += 32 / kTrsvCl) {
      uint4 v;
      if constexpr (sizeof(T) == 4) {
        v.x = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 0));
        v.y = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 1));
        v.z = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 2));
        v.w = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 3));
      } else {
        const double d0 = __shfl_sync(0xffffffffu, xk, pc * EP + 0);
        const double d1 = __shfl_sync(0xffffffffu, xk, pc * EP + 1);
        v.x = (uint32_t)__double2loint(d0);
        v.y = (uint32_t)__double2hiint(d0);
        v.z = (uint32_t)__double2loint(d1);
        v.w = (uint32_t)__double2hiint(d1);
      }
      st_async_16(rx + (uint32_t)(pc * 16), v, rb);
    }
    if (lane < rows) x[32 * k + lane] = (TOUT)xk;
    (void)w;
  }
  // ---- leave only when every x has landed here (no st.async still targets this CTA)
  if (tid == 0)
    for (int k = 0; k < nb; ++k) cl_wait(bar0 + 8 * k, err);
  __syncthreads();
  cl_sync();
}

// ------------------------------------------------------------ cluster solve, streamed tiles
// The same data flow where the row panels do not fit in the cluster's shared memory
// (n = 1000 in FP32: 2 MB of triangle against 1.8 MB).  The owner warp of block k
// needs M_kj only when x_j arrives, in a known order, so it streams the 32 x 32 tiles
// through a ring of kTrsvRing slots of its own (one bulk copy per tile row, completion
// on the slot's mbarrier), issued kTrsvRing dependencies ahead; the critical path is
// unchanged (one cluster hop plus two 32 x 32 products per block).
constexpr int kTrsvRing = 4;

// Shared memory of a CTA of the streamed solve (the largest owner count).
template <typename T>
__host__ __device__ inline size_t cls_smem(int n) {
  const int nb = (n + 31) / 32;
  const size_t nown = (size_t)((nb + kTrsvCl - 1) / kTrsvCl);
  const size_t head = ((size_t)32 * nb * sizeof(T) + 8 * (size_t)nb + 15) & ~(size_t)15;
  const size_t slot = (size_t)32 * ClPanel<T>::stride(32) * sizeof(T);
  return head + nown * kTrsvRing * 8 + nown * 1024 * sizeof(T) + nown * kTrsvRing * slot;
}

template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvClThreads)
    trsv_stream_kernel(const T* __restrict__ Q, int64_t ld, const T* __restrict__ D, int n,
                       const TIN* __restrict__ y, double yscale, TOUT* __restrict__ x, const int* done,
                       const int* jp, int64_t ys, int64_t xstr, int* err) {
  using P = ClPanel<T>;
  constexpr int TS = 32 + P::VE;   // ring row stride (P::stride(32))
  if (done && *done) return;   // uniform over the cluster: no CTA reaches a cluster barrier
  if (jp) {
    const int64_t j = *jp;
    y += j * ys;
    x += j * xstr;
  }
  extern __shared__ __align__(16) unsigned char cl_buf[];
  const int nb = (n + 31) >> 5;
  const uint32_t q = cl_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- layout: [x: 32 nb][bars: nb] (same offsets in every CTA: remote addresses are
  // mapped) [ring bars: nown x kTrsvRing][D of owned blocks][rings: nown x kTrsvRing x 32 x TS]
  T* xall = reinterpret_cast<T*>(cl_buf);
  uint64_t* bars = reinterpret_cast<uint64_t*>(cl_buf + (size_t)32 * nb * sizeof(T));
  unsigned char* cur = cl_buf + (((size_t)32 * nb * sizeof(T) + 8 * (size_t)nb + 15) & ~(size_t)15);
  const int nown = (nb - (int)q + kTrsvCl - 1) / kTrsvCl;   // blocks q, q + 8, ... below nb
  uint64_t* rbars = reinterpret_cast<uint64_t*>(cur);
  cur += (size_t)nown * kTrsvRing * 8;
  T* dblk = reinterpret_cast<T*>(cur);
  cur += (size_t)nown * 1024 * sizeof(T);
  T* ring = reinterpret_cast<T*>(cur);
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t xall0 = smem_u32(xall);
  __shared__ uint64_t load_bar;
  const uint32_t lbar = smem_u32(&load_bar);
  if (tid == 0) {
    for (int k = 0; k < nb; ++k) mbar_init(bar0 + 8 * k, 1);
    for (int e = 0; e < nown * kTrsvRing; ++e) mbar_init(smem_u32(rbars + e), 1);
    mbar_init(lbar, 1);
    fence_barrier_init();
    for (int k = 0; k < nb; ++k) mbar_arrive_expect_tx(bar0 + 8 * k, 32u * (uint32_t)sizeof(T));
  }
  // zero what the copies never cover: rows past the matrix in every slot of the last
  // block's ring, and (upper) the column tail of slot 0, which takes the partial last
  // column block as every block's first dependency
  const int tail_valid = n - 32 * (nb - 1);                                  // 1 .. 32
  const int tail_copied = (tail_valid + P::VE - 1) / P::VE * P::VE;
  for (int t = 0; t < nown; ++t) {
    const int k = (int)q + t * kTrsvCl;
    const int rows = min(32, n - 32 * k);
    T* rt = ring + (size_t)t * kTrsvRing * 32 * TS;
    for (int e = tid; e < kTrsvRing * (32 - rows) * 32; e += blockDim.x) {
      const int sl = e / ((32 - rows) * 32), r = rows + (e / 32) % (32 - rows), cc = e % 32;
      rt[((size_t)sl * 32 + r) * TS + cc] = T(0);
    }
    if (UPPER && tail_copied < 32)
      for (int e = tid; e < 32 * (32 - tail_copied); e += blockDim.x)
        rt[(size_t)(e / (32 - tail_copied)) * TS + tail_copied + e % (32 - tail_copied)] = T(0);
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) mbar_arrive_expect_tx(lbar, (uint32_t)(nown * 1024 * sizeof(T)));
    __syncwarp();
    if (lane < nown)
      bulk_load(smem_u32(dblk + (size_t)lane * 1024), D + (size_t)((int)q + lane * kTrsvCl) * 1024,
                1024u * (uint32_t)sizeof(T), lbar);
  }
  // every CTA's barriers are initialised before anyone sends
  cl_sync();
  if (warp < nown) {
    const int t = warp;
    const int k = (int)q + t * kTrsvCl;
    const int rows = min(32, n - 32 * k);
    T* rt = ring + (size_t)t * kTrsvRing * 32 * TS;
    const uint32_t rb0 = smem_u32(rbars + t * kTrsvRing);
    const int ndep = UPPER ? nb - 1 - k : k;
    // tile M_kj of dependency d into slot d % kTrsvRing: row r is Q[32k + r][32j ..]
    auto issue = [&](int d) {
      const int j = UPPER ? nb - 1 - d : d;
      const int valid = min(32, n - 32 * j);
      const uint32_t seg = (uint32_t)((valid + P::VE - 1) / P::VE * 16);
      const int sl = d % kTrsvRing;
      if (lane == 0) mbar_arrive_expect_tx(rb0 + 8 * sl, seg * (uint32_t)rows);
      __syncwarp();
      if (lane < rows)
        bulk_load(smem_u32(rt + ((size_t)sl * 32 + lane) * TS), Q + (size_t)(32 * k + lane) * ld + 32 * j, seg,
                  rb0 + 8 * sl);
    };
    int issued = min(kTrsvRing, ndep), landed = 0;
    for (int d = 0; d < issued; ++d) issue(d);
    T acc = (lane < rows) ? (T)((double)y[32 * k + lane] * yscale) : T(0);
    bool ok = mbar_wait(lbar, 0, err, DEV_TIMEOUT_FULL);
    for (int d = 0; d < ndep && ok; ++d) {
      const int j = UPPER ? nb - 1 - d : d;
      ok = mbar_wait(rb0 + 8 * (d % kTrsvRing), (uint32_t)(d / kTrsvRing) & 1u, err, DEV_TIMEOUT_FULL);
      if (!ok) break;
      landed = d + 1;
      ok = cl_wait(bar0 + 8 * j, err);
      if (!ok) break;
      const T* pr = rt + ((size_t)(d % kTrsvRing) * 32 + lane) * TS;
      const T* xj = xall + 32 * j;
      T s = T(0);
#pragma unroll
      for (int c = 0; c < 32; c += P::VE) {
        if constexpr (sizeof(T) == 4) {
          const float4 mv = *reinterpret_cast<const float4*>(pr + c);
          const float4 xv = *reinterpret_cast<const float4*>(xj + c);
          s += mv.x * xv.x + mv.y * xv.y + mv.z * xv.z + mv.w * xv.w;
        } else {
          const double2 mv = *reinterpret_cast<const double2*>(pr + c);
          const double2 xv = *reinterpret_cast<const double2*>(xj + c);
          s += mv.x * xv.x + mv.y * xv.y;
        }
      }
      acc -= s;
      __syncwarp();   // every lane has read the slot before it is refilled
      if (d + kTrsvRing < ndep) {
        issue(d + kTrsvRing);
        issued = d + kTrsvRing + 1;
      }
    }
    // after an expired wait: let the copies still in flight land (bounded) before leaving
    for (int d = landed; d < issued; ++d)
      mbar_wait(rb0 + 8 * (d % kTrsvRing), (uint32_t)(d / kTrsvRing) & 1u, err, DEV_TIMEOUT_FULL);
    // x_k = D_k^-1 y_k (lane r: sum_c D[c][r] y_c), then to every CTA of the cluster
    const T* dk = dblk + (size_t)t * 1024;
    T xa = T(0), xb = T(0);
#pragma unroll 8
    for (int c = 0; c < 32; c += 2) {
      xa += dk[c * 32 + lane] * __shfl_sync(0xffffffffu, acc, c);
      xb += dk[(c + 1) * 32 + lane] * __shfl_sync(0xffffffffu, acc, c + 1);
    }
    T xk = xa + xb;
    if (lane >= rows) xk = T(0);
    constexpr int EP = 16 / (int)sizeof(T);
    constexpr int PIECES = 32 / EP;
    const uint32_t dst = (uint32_t)(lane & (kTrsvCl - 1));
    const uint32_t rx = cl_map(xall0 + (uint32_t)(32 * k * sizeof(T)), dst);
    const uint32_t rbr = cl_map(bar0 + 8 * k, dst);
#pragma unroll
    for (int pc = lane / kTrsvCl; pc < PIECES; pc += 32 / kTrsvCl) {
      uint4 v;
      if constexpr (sizeof(T) == 4) {
        v.x = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 0));
        v.y = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 1));
        v.z = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 2));
        v.w = __float_as_uint(__shfl_sync(0xffffffffu, xk, pc * EP + 3));
      } else {
        const double d0 = __shfl_sync(0xffffffffu, xk, pc * EP + 0);
        const double d1 = __shfl_sync(0xffffffffu, xk, pc * EP + 1);
        v.x = (uint32_t)__double2loint(d0);
        v.y = (uint32_t)__double2hiint(d0);
        v.z = (uint32_t)__double2loint(d1);
        v.w = (uint32_t)__double2hiint(d1);
      }
      st_async_16(rx + (uint32_t)(pc * 16), v, rbr);
    }
    if (lane < rows) x[32 * k + lane] = (TOUT)xk;
  }
  // ---- leave only when every x has landed here (no st.async still targets this CTA)
  // and every tile copy issued here has completed
  if (tid == 0)
    for (int k = 0; k < nb; ++k) cl_wait(bar0 + 8 * k, err);
  __syncthreads();
  cl_sync();
}

template <typename T, typename TIN, typename TOUT, bool UPPER>
static cudaError_t launch_trsv_cluster(const T* Q, int64_t ld, const T* D, int n, const TIN* y, double yscale,
                                       TOUT* x, const int* done, cudaStream_t st, const int* jp, int64_t ys,
                                       int64_t xstr, int* err, size_t smem) {
  auto kern = trsv_cluster_kernel<T, TIN, TOUT, UPPER>;
  cudaError_t e = allow_dyn_smem(kern, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTrsvCl);
  cfg.blockDim = dim3(kTrsvClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTrsvCl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, Q, ld, D, n, y, yscale, x, done, jp, ys, xstr, err);
}

template <typename T, typename TIN, typename TOUT, bool UPPER>
static cudaError_t launch_trsv_stream(const T* Q, int64_t ld, const T* D, int n, const TIN* y, double yscale,
                                      TOUT* x, const int* done, cudaStream_t st, const int* jp, int64_t ys,
                                      int64_t xstr, int* err, size_t smem) {
  auto kern = trsv_stream_kernel<T, TIN, TOUT, UPPER>;
  cudaError_t e = allow_dyn_smem(kern, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTrsvCl);
  cfg.blockDim = dim3(kTrsvClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTrsvCl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, Q, ld, D, n, y, yscale, x, done, jp, ys, xstr, err);
}

// Largest per-CTA shared memory of the cluster solve (0 if it does not fit).
template <typename T>
static size_t cl_smem_max(bool upper, int n) {
  const int nb = (n + 31) / 32;
  if (nb > kTrsvCl * (kTrsvClThreads / 32)) return 0;   // at most one block per warp
  size_t mx = 0;
  for (int q = 0; q < kTrsvCl; ++q) mx = std::max(mx, cl_smem<T>(upper, n, q));
  return mx <= 200 * 1024 ? mx : 0;
}

template <typename T, typename TIN, typename TOUT>
cudaError_t launch_trsv(bool upper, const Tri<T>& f, const TIN* y, double yscale, TOUT* x,
                        const int* done, cudaStream_t st, const int* jp, int64_t ys, int64_t xstr) {
  if (f.n > 1024) return cudaErrorInvalidValue;
  // the cluster solve whenever its panels fit in shared memory (every CTA the same size)
  const size_t csm = cl_smem_max<T>(upper, (int)f.n);
  if (csm) {
    return upper ? launch_trsv_cluster<T, TIN, TOUT, true>(f.L, f.ld, f.DU, (int)f.n, y, yscale, x, done, st,
                                                          jp, ys, xstr, f.err, csm)
                 : launch_trsv_cluster<T, TIN, TOUT, false>(f.R, f.ld, f.DL, (int)f.n, y, yscale, x, done,
                                                           st, jp, ys, xstr, f.err, csm);
  }
  // past that, the cluster solve with streamed tiles (at most one block per warp)
  const int nbk = (int)((f.n + 31) / 32);
  const size_t ssm = cls_smem<T>((int)f.n);
  if (f.n > 32 && nbk <= kTrsvCl * (kTrsvClThreads / 32) && ssm <= 200 * 1024) {
    return upper ? launch_trsv_stream<T, TIN, TOUT, true>(f.L, f.ld, f.DU, (int)f.n, y, yscale, x, done, st, jp,
                                                         ys, xstr, f.err, ssm)
                 : launch_trsv_stream<T, TIN, TOUT, false>(f.R, f.ld, f.DL, (int)f.n, y, yscale, x, done, st,
                                                          jp, ys, xstr, f.err, ssm);
  }
  const size_t smem = TrsvSmem<T>::bytes;
  if (upper) {
    auto kern = trsv_kernel<T, TIN, TOUT, true>;
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kTrsvThreads, smem, st>>>(f.R, f.ld, f.DU, (int)f.n, y, yscale, x, done, jp, ys, xstr, f.err);
  } else {
    auto kern = trsv_kernel<T, TIN, TOUT, false>;
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kTrsvThreads, smem, st>>>(f.L, f.ld, f.DL, (int)f.n, y, yscale, x, done, jp, ys, xstr, f.err);
  }
  return cudaGetLastError();
}

#define LSQ_TRSV_INST(T, TIN, TOUT)                                                                  \
  template cudaError_t launch_trsv<T, TIN, TOUT>(bool, const Tri<T>&, const TIN*, double, TOUT*,  \
                                                 const int*, cudaStream_t, const int*, int64_t,   \
                                                 int64_t);
LSQ_TRSV_INST(float, float, float)
LSQ_TRSV_INST(float, double, float)
LSQ_TRSV_INST(float, float, double)
LSQ_TRSV_INST(float, double, double)
LSQ_TRSV_INST(double, double, double)
LSQ_TRSV_INST(double, float, double)
LSQ_TRSV_INST(double, double, float)
LSQ_TRSV_INST(double, float, float)

// ------------------------------------------------------------ preparation
__device__ __forceinline__ void prepare_r_body(const double* __restrict__ R, int64_t n, float* R32, float* L32,
                                               int64_t ld32, double* R64, double* L64, int64_t ld64, int64_t j) {
  for (int64_t i = threadIdx.x; i < ld32; i += blockDim.x) {
    const double v = (i <= j && i < n) ? R[j * n + i] : 0.0;   // R(i, j), upper
    R32[j * ld32 + i] = (float)v;
    if (i < n) L32[i * ld32 + j] = (float)v;                  // L(j, i) = R(i, j)
    else L32[j * ld32 + i] = 0.0f;                            // padding rows of L's column j
  }
  for (int64_t i = threadIdx.x; i < ld64; i += blockDim.x) {
    const double v = (i <= j && i < n) ? R[j * n + i] : 0.0;
    R64[j * ld64 + i] = v;
    if (i < n) L64[i * ld64 + j] = v;
    else L64[j * ld64 + i] = 0.0;
  }
}

__global__ void prepare_r_kernel(const double* __restrict__ R, int64_t n, float* R32, float* L32,
                                 int64_t ld32, double* R64, double* L64, int64_t ld64) {
  prepare_r_body(R, n, R32, L32, ld32, R64, L64, ld64, blockIdx.x);
}

// Inverse of the diagonal block k of the upper-triangular R (one warp per
// block): lane j forms column j of T^-1 by back substitution.  DU(i, j) at
// k*1024 + j*32 + i; DL = DU^T (the inverse of the diagonal block of R^T) at
// k*1024 + i*32 + j.
template <typename T>
__device__ __forceinline__ void dinv_body(const T* __restrict__ R, int64_t ld, int n, T* __restrict__ DU,
                                          T* __restrict__ DL, int k) {
  __shared__ T tb[32][33];
  const int lane = threadIdx.x;
  const int i0 = k * 32, w = min(32, n - i0);
  for (int c = 0; c < 32; ++c) tb[lane][c] = (lane < w && c < w) ? R[(size_t)(i0 + c) * ld + i0 + lane] : T(0);
  __syncwarp();
  T x[32];
#pragma unroll
  for (int i = 31; i >= 0; --i) {
    T t = (i == lane) ? T(1) : T(0);
#pragma unroll
    for (int c = i + 1; c < 32; ++c) t -= tb[i][c] * x[c];
    x[i] = (i < w && lane < w) ? t / tb[i][i] : T(0);
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    DU[(size_t)k * 1024 + lane * 32 + i] = x[i];
    DL[(size_t)k * 1024 + i * 32 + lane] = x[i];
  }
}

template <typename T>
__global__ void dinv_kernel(const T* __restrict__ R, int64_t ld, int n, T* __restrict__ DU,
                            T* __restrict__ DL) {
  dinv_body<T>(R, ld, n, DU, DL, blockIdx.x);
}

__device__ __forceinline__ void kappa_diag_body(const double* __restrict__ R, int64_t n, double* out) {
  __shared__ double mx[32], mn[32];
  double a = 0.0, b = INFINITY;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = fabs(R[i * n + i]);
    if (!(d < INFINITY)) bad = true;
    a = fmax(a, d);
    b = fmin(b, d);
  }
  if (bad) b = 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmin(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    mx[warp] = a;
    mn[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = fmax(a, mx[w]);
      b = fmin(b, mn[w]);
    }
    *out = (b > 0.0) ? a / b : INFINITY;
  }
}

__global__ void kappa_diag_kernel(const double* __restrict__ R, int64_t n, double* out) {
  kappa_diag_body(R, n, out);
}

cudaError_t launch_prepare_r(const double* R, int64_t n, Tri<float>* f32, Tri<double>* f64,
                             double* kappa_est, cudaStream_t st) {
  prepare_r_kernel<<<(unsigned)n, 256, 0, st>>>(R, n, const_cast<float*>(f32->R), const_cast<float*>(f32->L),
                                                f32->ld, const_cast<double*>(f64->R),
                                                const_cast<double*>(f64->L), f64->ld);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((n + 31) / 32);
  dinv_kernel<float><<<nb, 32, 0, st>>>(f32->R, f32->ld, (int)n, const_cast<float*>(f32->DU),
                                        const_cast<float*>(f32->DL));
  dinv_kernel<double><<<nb, 32, 0, st>>>(f64->R, f64->ld, (int)n, const_cast<double*>(f64->DU),
                                         const_cast<double*>(f64->DL));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (kappa_est) {
    kappa_diag_kernel<<<1, 256, 0, st>>>(R, n, kappa_est);
    e = cudaGetLastError();
  }
  return e;
}


// ============================================================ grouped (batched) forms
template <typename T, typename TIN, typename TOUT, bool UPPER>
__global__ void __launch_bounds__(kTrsvThreads)
    grouped_trsv_kernel(const GTrsv<T, TIN, TOUT>* __restrict__ tab) {
  const GTrsv<T, TIN, TOUT>& g = tab[blockIdx.x];
  if (g.done && *g.done) return;
  const TIN* y = g.y;
  TOUT* x = g.x;
  if (g.jp) {
    const int64_t j = *g.jp;
    y += j * g.ys;
    x += j * g.xstr;
  }
  __shared__ T xs[1024];
  extern __shared__ __align__(16) unsigned char trsv_buf[];
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) xs[i] = (T)((double)y[i] * g.yscale);
  __syncthreads();
  if (!block_trsv<T, UPPER>(g.M, g.ld, g.D, g.n, xs, trsv_buf, nullptr)) return;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) x[i] = (TOUT)xs[i];
}

template <typename T, typename TIN, typename TOUT>
cudaError_t launch_grouped_trsv(bool upper, const GTrsv<T, TIN, TOUT>* tab, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  const size_t smem = TrsvSmem<T>::bytes;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nprob, kTrsvThreads, smem, st>>>(tab);
    return cudaGetLastError();
  };
  return upper ? go(grouped_trsv_kernel<T, TIN, TOUT, true>) : go(grouped_trsv_kernel<T, TIN, TOUT, false>);
}
template cudaError_t launch_grouped_trsv<float, double, double>(bool, const GTrsv<float, double, double>*, int,
                                                                cudaStream_t);
template cudaError_t launch_grouped_trsv<float, float, float>(bool, const GTrsv<float, float, float>*, int,
                                                              cudaStream_t);
template cudaError_t launch_grouped_trsv<float, double, float>(bool, const GTrsv<float, double, float>*, int,
                                                               cudaStream_t);
template cudaError_t launch_grouped_trsv<float, float, double>(bool, const GTrsv<float, float, double>*, int,
                                                               cudaStream_t);
template cudaError_t launch_grouped_trsv<double, double, double>(bool, const GTrsv<double, double, double>*,
                                                                 int, cudaStream_t);

__global__ void grouped_prepare_r_kernel(const GPrepR* __restrict__ tab, const int* __restrict__ start, int nprob) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GPrepR& g = tab[p];
  prepare_r_body(g.R, g.n, const_cast<float*>(g.f32.R), const_cast<float*>(g.f32.L), g.f32.ld,
                 const_cast<double*>(g.f64.R), const_cast<double*>(g.f64.L), g.f64.ld, (int64_t)blockIdx.x - start[p]);
}

template <typename T>
__global__ void grouped_dinv_kernel(const GPrepR* __restrict__ tab, const int* __restrict__ start, int nprob) {
  const int p = group_of(start, nprob, blockIdx.x);
  const GPrepR& g = tab[p];
  const int k = blockIdx.x - start[p];
  if constexpr (sizeof(T) == 4)
    dinv_body<float>(g.f32.R, g.f32.ld, (int)g.n, const_cast<float*>(g.f32.DU), const_cast<float*>(g.f32.DL), k);
  else
    dinv_body<double>(g.f64.R, g.f64.ld, (int)g.n, const_cast<double*>(g.f64.DU), const_cast<double*>(g.f64.DL), k);
}

__global__ void grouped_kappa_kernel(const GPrepR* __restrict__ tab) {
  const GPrepR& g = tab[blockIdx.x];
  kappa_diag_body(g.R, g.n, g.kappa);
}

cudaError_t launch_grouped_prepare_r(const GPrepR* tab, const int* col_start, int64_t col_ctas,
                                     const int* blk_start, int64_t blk_ctas, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  grouped_prepare_r_kernel<<<(unsigned)col_ctas, 256, 0, st>>>(tab, col_start, nprob);
  grouped_dinv_kernel<float><<<(unsigned)blk_ctas, 32, 0, st>>>(tab, blk_start, nprob);
  grouped_dinv_kernel<double><<<(unsigned)blk_ctas, 32, 0, st>>>(tab, blk_start, nprob);
  grouped_kappa_kernel<<<(unsigned)nprob, 256, 0, st>>>(tab);
  return cudaGetLastError();
}

}  // namespace lsq
