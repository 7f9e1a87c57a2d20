// Double-double arithmetic on the FP64 pipe: a value hi + lo with |lo| <= ulp(hi)/2,
// about 106 significant bits.  Built from the error-free transformations: Knuth's
// TwoSum, Dekker's Fast2Sum (|a| >= |b|), the FMA form of TwoProduct (p = fl(a b),
// e = fma(a, b, -p) exactly), and the double-double sum and quotient of Dekker (1971)
// in the accurate form given by Joldes, Muller and Popescu (ACM TOMS 44, 2017).  The
// _rn intrinsics keep the compiler from contracting or reassociating any step.
#pragma once
#include <cuda_runtime.h>

namespace lsq {

struct DD {
  double hi, lo;
};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}

// (hi, lo) = a * b exactly
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

// a + b, both double-double (relative error about 3 * 2^-106)
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  double s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __dadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __dadd_rn(e, f);
  DD r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// acc + a * (zh + zl): the product a zh exactly, a zl rounded once (it sits 2^-53 below)
__device__ __forceinline__ DD dd_fma(DD acc, double a, double zh, double zl) {
  DD p;
  two_prod(a, zh, p.hi, p.lo);
  p.lo = __fma_rn(a, zl, p.lo);
  return dd_add(acc, p);
}

// (hi + lo) / d: q1 = fl(hi / d), then the remainder hi + lo - q1 d (formed with an exact
// product) divided once more
__device__ __forceinline__ DD dd_div_d(DD a, double d) {
  const double q1 = __ddiv_rn(a.hi, d);
  double p, e;
  two_prod(q1, d, p, e);
  double s, t;
  two_sum(a.hi, -p, s, t);
  t = __dsub_rn(t, e);
  t = __dadd_rn(t, a.lo);
  const double q2 = __ddiv_rn(__dadd_rn(s, t), d);
  DD r;
  fast_two_sum(q1, q2, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ DD dd_shfl_xor(DD v, int mask) {
  DD r;
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, mask);
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, mask);
  return r;
}

// sum over the warp; every lane gets the same value (dd_add is commutative: TwoSum's
// error term is the exact rounding error whatever the operand order)
__device__ __forceinline__ DD dd_warp_sum(DD v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dd_add(v, dd_shfl_xor(v, o));
  return v;
}

}  // namespace lsq
