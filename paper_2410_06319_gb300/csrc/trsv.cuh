// Block triangular solve on a shared-memory vector (used by the TRSV kernel
// and by the fused LSQR step).
//
// Blocks of 32 rows.  A block step is x_k = D_k^-1 y_k (D_k^-1 = inverse of the
// 32 x 32 diagonal block, formed once per R) by warp 0, then the rank-32
// update y_r -= sum_c M(r, i0 + c) x_c of the remaining rows by all threads.
// The update operands are contiguous column segments of the column-major
// matrix; they are staged into shared memory with cp.async in chunks of at
// most TR rows, NBUF buffers deep across chunks and steps, so the loads of the
// next chunks (and of the next D_k^-1) overlap the current one.
#pragma once
#include <cstddef>
#include <cstdint>

namespace lsq {

constexpr int kTrsvThreads = 1024;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared memory the solver needs: NBUF chunk buffers of 32 x TR elements and
// NBUF diagonal-inverse buffers of 32 x 32 elements (copies run NBUF-1 items ahead).
template <typename T>
struct TrsvSmem {
  static constexpr int TR = (sizeof(T) == 4) ? 512 : 256;   // rows per staged chunk
  static constexpr int NBUF = 3;
  static constexpr size_t bytes = (size_t)NBUF * 32 * TR * sizeof(T) + (size_t)NBUF * 1024 * sizeof(T);
};

// Solves in place on xs (shared, n entries): upper -> R x = y, lower -> L x = y.
// M is column-major with leading dimension ld (a multiple of 16 bytes / sizeof(T)),
// D holds the 1024-entry inverses of the diagonal blocks, `buf` is TrsvSmem<T>::bytes
// of shared memory.  Needs blockDim.x == kTrsvThreads.  Has no waits that can run
// out, so it always returns true (the signature matches solvers that do).
template <typename T, bool UPPER>
__device__ __forceinline__ bool block_trsv(const T* __restrict__ M, int64_t ld, const T* __restrict__ D,
                                           int n, T* xs, unsigned char* buf, int* /*err*/) {
  constexpr int TR = TrsvSmem<T>::TR;
  constexpr int NBUF = TrsvSmem<T>::NBUF;
  constexpr int VE = 16 / sizeof(T);                 // elements per 16-byte copy
  T* const base = reinterpret_cast<T*>(buf);
  auto chunk = [&](int sl) { return base + sl * 32 * TR; };
  auto dbuf = [&](int sl) { return base + NBUF * 32 * TR + sl * 1024; };
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (n + 31) >> 5;
  // work items: (step, row chunk); a step with no remaining rows still has one
  // (empty) item so that its diagonal block is solved.
  auto rows_of = [&](int step, int& lo, int& hi) {
    const int k = UPPER ? nb - 1 - step : step;
    const int i0 = k * 32, w = min(32, n - i0);
    if (UPPER) {
      lo = 0;
      hi = i0;
    } else {
      lo = i0 + w;
      hi = n;
    }
  };
  auto nchunks = [&](int step) {
    int lo, hi;
    rows_of(step, lo, hi);
    return hi > lo ? (hi - lo + TR - 1) / TR : 1;
  };
  // issue the async copies of item (step, ci) into buffer slot `sl`
  auto issue = [&](int step, int ci, int sl) {
    const int k = UPPER ? nb - 1 - step : step;
    const int i0 = k * 32, w = min(32, n - i0);
    int lo, hi;
    rows_of(step, lo, hi);
    if (ci == 0) {  // the diagonal inverse of the step travels with its first chunk
      for (int e = tid * VE; e < 1024; e += blockDim.x * VE) cp_async16(dbuf(sl) + e, D + (size_t)k * 1024 + e);
    }
    const int r0 = lo + ci * TR, r1 = min(hi, r0 + TR);
    if (r1 > r0) {
      const int a0 = r0 & ~(VE - 1);                  // 16-byte aligned start
      const int segs = (r1 - a0 + VE - 1) / VE;       // 16-byte pieces per column
      for (int e = tid; e < w * segs; e += blockDim.x) {
        const int c = e / segs, sgi = e % segs;
        cp_async16(chunk(sl) + c * TR + sgi * VE, M + (size_t)(i0 + c) * ld + a0 + sgi * VE);
      }
    }
    cp_async_commit();
  };
  // the item sequence (step, chunk), advanced in order
  auto advance = [&](int& st, int& c) {
    if (++c >= nchunks(st)) {
      ++st;
      c = 0;
    }
  };
  // prefetch the first NBUF-1 items
  int pst = 0, pci = 0, psl = 0;
  for (int q = 0; q < NBUF - 1; ++q) {
    if (pst < nb) {
      issue(pst, pci, psl);
      advance(pst, pci);
    } else {
      cp_async_commit();
    }
    psl = (psl + 1) % NBUF;
  }
  int step = 0, ci = 0, sl = 0;
  while (step < nb) {
    const int k = UPPER ? nb - 1 - step : step;
    const int i0 = k * 32, w = min(32, n - i0);
    // keep NBUF-1 items in flight
    if (pst < nb) {
      issue(pst, pci, psl);
      advance(pst, pci);
    } else {
      cp_async_commit();
    }
    psl = (psl + 1) % NBUF;
    cp_async_wait<NBUF - 1>();
    __syncthreads();
    if (ci == 0) {   // diagonal block: x_k = D_k^-1 y_k
      if (warp == 0) {
        const T* dk = dbuf(sl);
        T acc = T(0);
#pragma unroll 8
        for (int c = 0; c < w; ++c) acc += dk[c * 32 + lane] * xs[i0 + c];
        __syncwarp();
        if (lane < w) xs[i0 + lane] = acc;
      }
      __syncthreads();
    }
    int lo, hi;
    rows_of(step, lo, hi);
    const int r0 = lo + ci * TR, r1 = min(hi, r0 + TR);
    if (r1 > r0) {
      const int a0 = r0 & ~(VE - 1);
      const T* ch = chunk(sl);
      // TR rows, 1024 threads: 1024 / TR threads per row share the 32 columns
      constexpr int TPR = 1024 / TR;
      const int rr = tid / TPR, part = tid % TPR;
      const int r = r0 + rr;
      T acc = T(0);
      if (r < r1) {
#pragma unroll 8
        for (int c = part; c < w; c += TPR) acc += ch[c * TR + (r - a0)] * xs[i0 + c];
      }
      if (TPR > 1) {
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, TPR);
      }
      if (r < r1 && part == 0) xs[r] -= acc;
    }
    __syncthreads();
    advance(step, ci);
    sl = (sl + 1) % NBUF;
  }
  cp_async_wait<0>();
  return true;
}

}  // namespace lsq
