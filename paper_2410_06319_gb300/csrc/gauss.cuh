// The sketch matrix G of Omega = s^-1/2 fl_s(G), generated on the fly.
//
// Definition (Sec. 2 Gaussian embedding with N(0, 1/s) entries; Sec. 5 uses
// Omega = (4n)^-1/2 G): G[i, j] for sketch row i and data row j is
//   (x0, x1, x2, x3) = Philox4x32-10(counter = (j>>2, i, j>>34, 0),
//                                    key = (seed lo, seed hi))        [SC'11]
//   (a, b) = (x0, x1) if j%4 < 2 else (x2, x3)
//   U1 = (a + 1) 2^-32,  U2 = b 2^-32,  R = sqrt(-2 ln U1)
//   G = R cos(2 pi U2) for even j, R sin(2 pi U2) for odd j; G = +0 if a = 2^32-1
// with ln and (cos, sin)(2 pi U2) evaluated by the fixed IEEE double sequences
// spec_ln_u1 / spec_cos_sin_2pi below (no fused multiply-add).  The operand
// used by a sketch in precision u_s is fl_s(G), round to nearest even.
//
// Evaluation on GB300: FP64 is a slow pipe, so G is first evaluated in FP32
// (fast_*) with a relative error below 2^-20.4 against the FP64 definition;
// if both ends of [g32 (1 - 2^-19), g32 (1 + 2^-19)] round to the same u_s
// value, that value is fl_s(G) exactly.  Otherwise the FP64 definition is
// evaluated and rounded (round-to-odd to FP32, then to u_s: a single
// rounding of the FP64 value).  The result is bit-identical to rounding the
// FP64 definition directly.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace lsq {

enum SFmt : int { FMT_F64 = 0, FMT_F32 = 1, FMT_F16 = 2, FMT_BF16 = 3, FMT_E4M3 = 4, FMT_BF16X3 = 5 };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Counter of the Philox call serving sketch row i, data rows 4q .. 4q+3.
__device__ __forceinline__ uint4 gauss_counter(uint64_t q, uint32_t i) {
  return make_uint4((uint32_t)q, i, (uint32_t)(q >> 32), 0u);
}

// ------------------------------------------------------------ FP64 definition
__device__ __forceinline__ double spec_ln_u1(uint32_t a) {
  // U1 = 2^e f, f in [sqrt(1/2), sqrt(2)); ln f = 2 atanh(z), z = (f-1)/(f+1),
  // series 2z (1 + w/3 + ... + w^11/23), w = z^2, Horner with separate * and +.
  const double u1 = (double)((uint64_t)a + 1ull) * 0x1p-32;
  const long long bits = __double_as_longlong(u1);
  double e = (double)((int)((bits >> 52) & 0x7FF) - 1023);
  double f = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  if (f > 1.4142135623730951) {
    f = __dmul_rn(f, 0.5);
    e = __dadd_rn(e, 1.0);
  }
  const double z = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
  const double w = __dmul_rn(z, z);
  double p = 1.0 / 23.0;
  p = __dadd_rn(1.0 / 21.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 19.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 17.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 15.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 13.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 11.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 9.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 7.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 5.0, __dmul_rn(w, p));
  p = __dadd_rn(1.0 / 3.0, __dmul_rn(w, p));
  const double z2 = __dmul_rn(z, 2.0);
  const double lnf = __dadd_rn(z2, __dmul_rn(z2, __dmul_rn(w, p)));
  return __dadd_rn(__dmul_rn(e, 0.6931471805599453), lnf);
}

__device__ __forceinline__ void spec_cos_sin_2pi(uint32_t b, double& c, double& s) {
  // 4 U2 = q + r, r moved to [-1/2, 1/2); phi = r (pi/2); Taylor series of sin
  // and cos to phi^21 / phi^20 (Horner, separate * and +); rotate by q.
  uint32_t q = b >> 30;
  int32_t rb = (int32_t)(b & 0x3FFFFFFFu);
  if (rb >= (1 << 29)) {
    rb -= (1 << 30);
    q = (q + 1u) & 3u;
  }
  const double r = (double)rb * 0x1p-30;
  const double phi = __dmul_rn(r, 1.5707963267948966);
  const double w = __dmul_rn(phi, phi);
  double ps = 1.0 / 51090942171709440000.0;           // +1/21!
  ps = __dadd_rn(-1.0 / 121645100408832000.0, __dmul_rn(w, ps));
  ps = __dadd_rn(1.0 / 355687428096000.0, __dmul_rn(w, ps));
  ps = __dadd_rn(-1.0 / 1307674368000.0, __dmul_rn(w, ps));
  ps = __dadd_rn(1.0 / 6227020800.0, __dmul_rn(w, ps));
  ps = __dadd_rn(-1.0 / 39916800.0, __dmul_rn(w, ps));
  ps = __dadd_rn(1.0 / 362880.0, __dmul_rn(w, ps));
  ps = __dadd_rn(-1.0 / 5040.0, __dmul_rn(w, ps));
  ps = __dadd_rn(1.0 / 120.0, __dmul_rn(w, ps));
  ps = __dadd_rn(-1.0 / 6.0, __dmul_rn(w, ps));
  const double sphi = __dadd_rn(phi, __dmul_rn(phi, __dmul_rn(w, ps)));
  double pc = 1.0 / 2432902008176640000.0;            // +1/20!
  pc = __dadd_rn(-1.0 / 6402373705728000.0, __dmul_rn(w, pc));
  pc = __dadd_rn(1.0 / 20922789888000.0, __dmul_rn(w, pc));
  pc = __dadd_rn(-1.0 / 87178291200.0, __dmul_rn(w, pc));
  pc = __dadd_rn(1.0 / 479001600.0, __dmul_rn(w, pc));
  pc = __dadd_rn(-1.0 / 3628800.0, __dmul_rn(w, pc));
  pc = __dadd_rn(1.0 / 40320.0, __dmul_rn(w, pc));
  pc = __dadd_rn(-1.0 / 720.0, __dmul_rn(w, pc));
  pc = __dadd_rn(1.0 / 24.0, __dmul_rn(w, pc));
  pc = __dadd_rn(-1.0 / 2.0, __dmul_rn(w, pc));
  const double cphi = __dadd_rn(1.0, __dmul_rn(w, pc));
  switch (q) {
    case 0: c = cphi; s = sphi; break;
    case 1: c = -sphi; s = cphi; break;
    case 2: c = -cphi; s = -sphi; break;
    default: c = sphi; s = -cphi; break;
  }
}

__device__ __forceinline__ void spec_gauss_pair(uint32_t a, uint32_t b, double& ge, double& go) {
  if (a == 0xFFFFFFFFu) {
    ge = 0.0;
    go = 0.0;
    return;
  }
  const double rad = __dsqrt_rn(__dmul_rn(-2.0, spec_ln_u1(a)));
  double c, s;
  spec_cos_sin_2pi(b, c, s);
  ge = __dmul_rn(rad, c);
  go = __dmul_rn(rad, s);
}

// ------------------------------------------------------------ FP32 evaluation
// Relative error against the FP64 definition, first order: ln U1 <= 12 ulp
// (conversion of U1 or 1 - U1: 1 ulp, amplified <= 2.9x where |ln U1| >= 0.35;
// the quotient z: f + 1 rounded plus a 2-ulp __fdividef; series rounding and
// truncation < 2 ulp; e ln2 + ln f with cancellation <= 2x), so the radius is
// within 6.5 ulp; the reduced angle is within 2.5 ulp (30-bit r converted,
// pi/2 rounded, one product) and sin/cos within 4.5 ulp; the final product adds
// 1 ulp.  Total 12 ulp = 2^-20.4; kFastRelBound = 2^-19 leaves a 2.6x margin.
constexpr float kFastRelBound = 0x1p-19f;

// Integer -> FP32 conversions and the rounding to u_s in the FP32 path are
// written with integer and FMA-pipe instructions: on GB300 the conversion
// instructions share the narrow FP64 pipe.  The values are the same as the
// conversions' (round to nearest even).
//
// x < 2^32 -> RN(x): both 16-bit halves are exact in FP32, one FMA rounds once.
__device__ __forceinline__ float u32_to_f32_rn(uint32_t x) {
  const float hi = __uint_as_float(0x4B000000u | (x >> 16)) - 8388608.0f;
  const float lo = __uint_as_float(0x4B000000u | (x & 0xFFFFu)) - 8388608.0f;
  return fmaf(hi, 65536.0f, lo);
}
// small non-negative integer field f (f < 2^23) minus `bias`, exactly
__device__ __forceinline__ float field_minus(uint32_t f, float bias) {
  return (__uint_as_float(0x4B000000u | f) - 8388608.0f) - bias;
}

__device__ __forceinline__ float fast_ln_u1(uint32_t a) {
  float z, e;
  if (a >= 0xB504F334u) {  // U1 > sqrt(1/2): ln(1 - V) with V = 1 - U1 exact in integers
    const float V = u32_to_f32_rn(~a) * 0x1p-32f;
    z = __fdividef(-V, 2.0f - V);
    e = 0.0f;
  } else {
    const float u = u32_to_f32_rn(a + 1u) * 0x1p-32f;
    const uint32_t ub = __float_as_uint(u);
    float f = __uint_as_float((ub & 0x007FFFFFu) | 0x3F800000u);
    e = field_minus(ub >> 23, 127.0f);   // exponent of u (u is normal)
    if (f > 1.41421356f) {
      f *= 0.5f;
      e += 1.0f;
    }
    z = __fdividef(f - 1.0f, f + 1.0f);
  }
  const float w = z * z;
  float p = 1.0f / 13.0f;
  p = fmaf(w, p, 1.0f / 11.0f);
  p = fmaf(w, p, 1.0f / 9.0f);
  p = fmaf(w, p, 1.0f / 7.0f);
  p = fmaf(w, p, 1.0f / 5.0f);
  p = fmaf(w, p, 1.0f / 3.0f);
  const float z2 = 2.0f * z;
  const float lnf = fmaf(z2 * w, p, z2);
  return fmaf(e, 0.693147180559945f, lnf);
}

__device__ __forceinline__ void fast_cos_sin_2pi(uint32_t b, float& c, float& s) {
  uint32_t q = b >> 30;
  int32_t rb = (int32_t)(b & 0x3FFFFFFFu);
  if (rb >= (1 << 29)) {
    rb -= (1 << 30);
    q = (q + 1u) & 3u;
  }
  const float rm = u32_to_f32_rn((uint32_t)(rb < 0 ? -rb : rb));   // RN(|rb|), |rb| <= 2^29
  const float phi = ((rb < 0 ? -rm : rm) * 0x1p-30f) * 1.57079632679489662f;
  const float w = phi * phi;
  float ps = 1.0f / 6227020800.0f;
  ps = fmaf(w, ps, -1.0f / 39916800.0f);
  ps = fmaf(w, ps, 1.0f / 362880.0f);
  ps = fmaf(w, ps, -1.0f / 5040.0f);
  ps = fmaf(w, ps, 1.0f / 120.0f);
  ps = fmaf(w, ps, -1.0f / 6.0f);
  const float sphi = fmaf(phi * w, ps, phi);
  float pc = 1.0f / 479001600.0f;
  pc = fmaf(w, pc, -1.0f / 3628800.0f);
  pc = fmaf(w, pc, 1.0f / 40320.0f);
  pc = fmaf(w, pc, -1.0f / 720.0f);
  pc = fmaf(w, pc, 1.0f / 24.0f);
  pc = fmaf(w, pc, -0.5f);
  const float cphi = fmaf(w, pc, 1.0f);
  const bool swap = (q & 1u) != 0;
  const float cc = swap ? sphi : cphi;
  const float ss = swap ? cphi : sphi;
  c = (q == 1u || q == 2u) ? -cc : cc;
  s = (q >= 2u) ? -ss : ss;
}

// ------------------------------------------------------------ rounding to u_s
template <int FMT>
__device__ __forceinline__ uint32_t round_f32(float x) {
  if constexpr (FMT == FMT_F16) {
    return (uint32_t)__half_as_ushort(__float2half_rn(x));
  } else if constexpr (FMT == FMT_BF16) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
  } else {
    return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
  }
}

// Single rounding of an FP64 value: round to odd into FP32 (24 bits, at least
// two more than every target), then round to nearest even into the target.
template <int FMT>
__device__ __forceinline__ uint32_t round_f64(double g) {
  float t = __double2float_rz(g);
  if ((double)t != g) t = __uint_as_float(__float_as_uint(t) | 1u);
  return round_f32<FMT>(t);
}

template <int FMT>
__device__ __forceinline__ double bits_to_double(uint32_t v) {
  if constexpr (FMT == FMT_F16) {
    return (double)__half2float(__ushort_as_half((unsigned short)v));
  } else if constexpr (FMT == FMT_BF16) {
    return (double)__bfloat162float(__ushort_as_bfloat16((unsigned short)v));
  } else {
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)v, __NV_E4M3);
    return (double)__half2float(__half(hr));
  }
}

template <int FMT>
__device__ __forceinline__ float bits_to_float(uint32_t v) {
  if constexpr (FMT == FMT_F16) {
    return __half2float(__ushort_as_half((unsigned short)v));
  } else if constexpr (FMT == FMT_BF16) {
    return __uint_as_float(v << 16);
  } else {
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)v, __NV_E4M3);
    return __half2float(__half(hr));
  }
}

// Rounds one FP32 estimate g to u_s; returns false when the FP64 definition is
// needed.  The true value lies within d = 2^-19 |g| of g, which is below 32
// FP32 ulps of g; if the nearest rounding midpoint of u_s (the FP32 pattern
// whose discarded low bits are exactly one half) is more than 32 ulps away,
// every value in [g - d, g + d] rounds as g does.  Binade changes within the
// interval do not matter: the format's values at a power of two are exact.
// Normal range of u_s only (g below it, or u_s overflow, falls back); `out` is
// always a finite pattern of the format's width (callers pack it, and the
// deferred sketch multiplies with it before correcting): fl_s(g), or signed zero
// below the normal range.
template <int FMT>
__device__ __forceinline__ bool round_checked(float g, uint32_t& out) {
  const uint32_t b = __float_as_uint(g);
  const uint32_t sg = b >> 31, mag = b & 0x7FFFFFFFu;
  if constexpr (FMT == FMT_BF16) {   // 7 fraction bits: 16 low bits dropped
    const int off = (int)(mag & 0xFFFFu) - 0x8000;
    out = (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
    return (off > 32 || off < -32) && mag >= 0x00800000u;
  } else if constexpr (FMT == FMT_F16) {   // 10 fraction bits, normal for |g| >= 2^-14
    if (mag < 0x38800000u) {   // below the normal range: signed zero, exact value later
      out = sg << 15;
      return false;
    }
    const int off = (int)(mag & 0x1FFFu) - 0x1000;
    const uint32_t r = mag + 0xFFFu + ((mag >> 13) & 1u);
    out = ((sg << 15) | ((r >> 13) - (112u << 10))) & 0xFFFFu;
    return (off > 32 || off < -32) && r < 0x47800000u;
  } else {   // E4M3: 3 fraction bits, normal for 2^-6 <= |g|, finite below 2^8 here
    if (mag < 0x3C800000u) {   // below the normal range: signed zero, exact value later
      out = sg << 7;
      return false;
    }
    const int off = (int)(mag & 0xFFFFFu) - 0x80000;
    const uint32_t r = mag + 0x7FFFFu + ((mag >> 20) & 1u);
    out = ((sg << 7) | ((r >> 20) - (120u << 3))) & 0xFFu;
    return (off > 32 || off < -32) && r < 0x43800000u;
  }
}

// FP32 evaluation of one (a, b) word pair; false when the FP64 definition is
// needed for either entry (near a rounding boundary of u_s, or U1 = 1).
template <int FMT>
__device__ __forceinline__ bool gauss_pair_fast(uint32_t a, uint32_t b, uint32_t& be, uint32_t& bo) {
  const float rad = __fsqrt_rn(-2.0f * fast_ln_u1(a));
  float c, s;
  fast_cos_sin_2pi(b, c, s);
  const bool oke = round_checked<FMT>(rad * c, be);
  const bool oko = round_checked<FMT>(rad * s, bo);
  return oke && oko && a != 0xFFFFFFFFu;
}

// The FP64 definition, rounded once into u_s.
template <int FMT>
__device__ __forceinline__ void gauss_pair_slow(uint32_t a, uint32_t b, uint32_t& be, uint32_t& bo) {
  double ge, go;
  spec_gauss_pair(a, b, ge, go);
  be = round_f64<FMT>(ge);
  bo = round_f64<FMT>(go);
}

// fl_s(G) bits of the two entries served by one (a, b) word pair.
template <int FMT>
__device__ __forceinline__ void gauss_pair_bits(uint32_t a, uint32_t b, uint32_t& be, uint32_t& bo) {
  if (!gauss_pair_fast<FMT>(a, b, be, bo)) gauss_pair_slow<FMT>(a, b, be, bo);
}

}  // namespace lsq
