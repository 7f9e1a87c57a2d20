// Exact rounding of FP64 values into the sketch formats on integer units
// (Sec. 3.2's A_s = fl_s(2^k A); the three-term BF16 split hi + lo + lo2).
//
// GB300's FP64 pipe, and FP64 conversions, are narrow.  Rounding an FP64 value
// to a format with P significant bits is exact integer arithmetic on its
// 53-bit significand as long as the result lies in the format's normal range,
// so the cast pass does that and leaves only zeros' signs and out-of-range
// values (subnormal results, overflow, non-finite input) to the FP64
// definition.  Plain C++ when compiled without nvcc, so a host harness can
// check it bit for bit against the oracle.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define LSQ_HD __host__ __device__ __forceinline__
#else
#define LSQ_HD inline
#endif

namespace lsq {

LSQ_HD int clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// Formats: MB fraction bits, normal exponents [EMIN, EMAX], bias, width.
struct EncBF16 {
  static constexpr int MB = 7, EMIN = -126, EMAX = 127, BIAS = 127, W = 16;
};
struct EncF16 {
  static constexpr int MB = 10, EMIN = -14, EMAX = 15, BIAS = 15, W = 16;
};
struct EncE4M3 {
  // the top binade (2^8 .. 448) is left to the FP64 definition and its saturation
  static constexpr int MB = 3, EMIN = -6, EMAX = 7, BIAS = 7, W = 8;
};
struct EncF32 {
  static constexpr int MB = 23, EMIN = -126, EMAX = 127, BIAS = 127, W = 32;
};

// Rounds a * 2^sc (a > 0) to MB + 1 significant bits, ties to even, and encodes
// the magnitude.  Returns false when the rounded value's exponent leaves
// [EMIN, EMAX].  `rounded` receives the rounded magnitude on the scale of a,
// so a - rounded is exact.
template <class F>
LSQ_HD bool rn_encode(uint64_t a, int sc, uint32_t& bits, uint64_t& rounded) {
  const int L = 63 - clz64(a);
  int e = L + sc;
  if (e < F::EMIN || e > F::EMAX) return false;
  uint32_t mant;
  if (L <= F::MB) {
    rounded = a;
    mant = (uint32_t)((a << (F::MB - L)) & ((1ull << F::MB) - 1));
  } else {
    const int sh = L - F::MB;
    uint64_t q = a >> sh;
    const uint64_t rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    rounded = q << sh;
    if (q >> (F::MB + 1)) {   // carried into the next binade
      q >>= 1;
      ++e;
      if (e > F::EMAX) return false;
    }
    mant = (uint32_t)(q & ((1ull << F::MB) - 1));
  }
  bits = ((uint32_t)(e + F::BIAS) << F::MB) | mant;
  return true;
}

// fl(sign * a * 2^sc), a > 0: the format's bit pattern.
template <class F>
LSQ_HD bool enc_term(uint32_t sg, uint64_t a, int sc, uint32_t& bits, uint64_t& rounded) {
  if (!rn_encode<F>(a, sc, bits, rounded)) return false;
  bits |= sg << (F::W - 1);
  return true;
}

// The terms of v = 2^k * x (x given by its FP64 bits u) in format F: t[0] =
// fl(v), and with SPLIT3 also t[1] = fl(v - t[0]), t[2] = fl(v - t[0] - t[1])
// (differences exact).  False when some term needs the FP64 definition.
template <class F, bool SPLIT3>
LSQ_HD bool cast_terms_int(uint64_t u, int k, uint32_t (&t)[3]) {
  const uint32_t sg = (uint32_t)(u >> 63);
  t[0] = t[1] = t[2] = 0;
  if ((u << 1) == 0) {                     // fl(+-0) = +-0; the differences are +0
    t[0] = sg << (F::W - 1);
    return true;
  }
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return false;  // subnormal or non-finite input
  const uint64_t a = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sc = E - 1075 + k;
  uint64_t rd;
  if (!enc_term<F>(sg, a, sc, t[0], rd)) return false;
  if (SPLIT3) {
    const int64_t d1 = (int64_t)a - (int64_t)rd;   // v - hi
    if (d1 == 0) return true;
    const uint32_t s1 = sg ^ (d1 < 0 ? 1u : 0u);
    const uint64_t a1 = (uint64_t)(d1 < 0 ? -d1 : d1);
    uint64_t rd1;
    if (!enc_term<F>(s1, a1, sc, t[1], rd1)) return false;
    const int64_t d2 = (int64_t)a1 - (int64_t)rd1;  // v - hi - lo
    if (d2 == 0) return true;
    const uint32_t s2 = s1 ^ (d2 < 0 ? 1u : 0u);
    uint64_t rd2;
    if (!enc_term<F>(s2, (uint64_t)(d2 < 0 ? -d2 : d2), sc, t[2], rd2)) return false;
  }
  return true;
}

}  // namespace lsq
