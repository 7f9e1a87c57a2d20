// Exact rounding of FP64 values into the sketch formats on integer units
// (Sec. 3.2's A_s = fl_s(2^k A)), and the BF16X3 operand: y = fl32(2^k A)
// carried as its exact three-term BF16 split hi + lo + lo2.
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
#include <cstring>

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

// t[0] = fl(v), v = 2^k * x (x given by its FP64 bits u) in format F; t[1] = t[2]
// = 0.  False when the result needs the FP64 definition (subnormal or
// overflowing result, subnormal or non-finite input).
template <class F>
LSQ_HD bool cast_terms_int(uint64_t u, int k, uint32_t (&t)[3]) {
  const uint32_t sg = (uint32_t)(u >> 63);
  t[0] = t[1] = t[2] = 0;
  if ((u << 1) == 0) {                     // fl(+-0) = +-0
    t[0] = sg << (F::W - 1);
    return true;
  }
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return false;  // subnormal or non-finite input
  const uint64_t a = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint64_t rd;
  return enc_term<F>(sg, a, E - 1075 + k, t[0], rd);
}

// fl32(x) for x given by its FP64 bits, when the result is a normal FP32 number or an
// infinity reached by rounding (biased FP64 exponent 897 .. 1150): round the 53-bit
// significand at bit 29 to nearest even by one 64-bit add (a carry out of the fraction
// moves into the exponent, up to the infinity past FP32's largest value), then rebias
// the exponent.  False otherwise (zero, subnormal results, non-finite x).
LSQ_HD bool f64_to_f32_bits(uint64_t u, uint32_t& out) {
  const uint32_t e = (uint32_t)(u >> 52) & 0x7FFu;
  if (e < 897u || e > 1150u) return false;
  const uint64_t r = u + 0x0FFFFFFFull + ((u >> 29) & 1ull);
  const uint32_t mag = (uint32_t)(((r >> 29) & 0x3FFFFFFFFull) - (896ull << 23));
  out = ((uint32_t)(u >> 32) & 0x80000000u) | mag;
  return true;
}

// fl32(2^k x) by f64_to_f32_bits on the exponent-shifted bits, for normal x with 2^k x
// a normal FP64 number (then 2^k x is exact in FP64).  False otherwise.
LSQ_HD bool f64_scaled_to_f32_bits(uint64_t u, int k, uint32_t& out) {
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF || e + k <= 0 || e + k >= 0x7FF) return false;
  return f64_to_f32_bits(u + ((uint64_t)(int64_t)k << 52), out);
}

// ---------------------------------------------------------------- BF16X3
LSQ_HD float f32_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, 4);
  return f;
#endif
}
LSQ_HD uint32_t bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
#endif
}
LSQ_HD float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

// fl_bf16 of a finite FP32 value given by its bits, ties to even.  BF16 keeps
// FP32's sign and exponent fields, so rounding away the low 16 bits of the
// pattern rounds the value, on the subnormal grid too; a carry out of the
// fraction moves into the exponent.
LSQ_HD uint32_t bf16_rn(uint32_t f) { return (f + 0x7FFFu + ((f >> 16) & 1u)) >> 16; }

// The split of y (FP32 bits): hi = fl_bf16(y), lo = fl_bf16(y - hi), lo2 =
// fl_bf16(y - hi - lo).  Each difference is an exact FP32 subtraction (the
// operands are within a factor of two of each other), and y - hi - lo has at
// most eight significant bits, so hi + lo + lo2 = y unless lo2 lies below
// BF16's normal range.
LSQ_HD void split3_f32(uint32_t y, uint32_t (&t)[3]) {
  t[0] = bf16_rn(y);
  const float r1 = sub_rn(f32_of(y), f32_of(t[0] << 16));
  t[1] = bf16_rn(bits_of(r1));
  const float r2 = sub_rn(r1, f32_of(t[1] << 16));
  t[2] = bf16_rn(bits_of(r2));
}

// fl32(2^k x) from a = fl32(x) (FP32 bits): 2^k a, exact when |a| and |2^k a|
// both lie in [2^-125, 2^128) -- x was then rounded on the normal grid and
// scaling by a power of two commutes with that rounding.  False otherwise
// (zero, subnormal or near-subnormal, non-finite).
LSQ_HD bool f32_scale_exact(uint32_t a, int k, uint32_t& y) {
  const int ef = (int)((a >> 23) & 0xFFu);
  const int es = ef + k;
  if (ef < 2 || ef > 254 || es < 2 || es > 254) return false;
  y = a + ((uint32_t)k << 23);
  return true;
}

}  // namespace lsq
