// Host harness for csrc/cast.cuh: reads "fmt" then lines "u_hex k" (FP64 bits
// and a power-of-two exponent) and prints "ok t0 t1 t2" (hex bit patterns).
// bf16, f16, e4m3, f32: ok = the integer rounding of 2^k * x into fmt took it.
// f32fast: the one-add FP64 -> FP32 rounding (k ignored).
// bf16x3: the three BF16 terms of y = fl32(2^k x), formed as the kernels do --
// from a = fl32(x) by a power-of-two scaling where that is exact (ok = 1), else
// from x itself (integer rounding, else the host's FP64 -> FP32 conversion).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "cast.cuh"

template <class F>
static void run() {
  unsigned long long u;
  int k;
  while (std::scanf("%llx %d", &u, &k) == 2) {
    uint32_t t[3];
    const bool ok = lsq::cast_terms_int<F>((uint64_t)u, k, t);
    std::printf("%d %x %x %x\n", ok ? 1 : 0, t[0], t[1], t[2]);
  }
}

static void run_bf16x3() {
  unsigned long long u;
  int k;
  while (std::scanf("%llx %d", &u, &k) == 2) {
    double x;
    std::memcpy(&x, &u, 8);
    const uint32_t a = lsq::bits_of((float)x);
    uint32_t y;
    const bool fast = lsq::f32_scale_exact(a, k, y);
    if (!fast) {   // the kernels' route from the FP64 value: one-add, integer, then the FP64 definition
      uint32_t t1[3];
      if (!lsq::f64_scaled_to_f32_bits((uint64_t)u, k, y))
        y = lsq::cast_terms_int<lsq::EncF32>((uint64_t)u, k, t1) ? t1[0] : lsq::bits_of((float)std::ldexp(x, k));
    }
    uint32_t t[3];
    lsq::split3_f32(y, t);
    std::printf("%d %x %x %x\n", fast ? 1 : 0, t[0], t[1], t[2]);
  }
}

// f32fast: the one-add rounding of f64_to_f32_bits (ok = it took the value)
static void run_f32fast() {
  unsigned long long u;
  int k;
  while (std::scanf("%llx %d", &u, &k) == 2) {
    uint32_t b = 0;
    const bool ok = lsq::f64_to_f32_bits((uint64_t)u, b);
    std::printf("%d %x 0 0\n", ok ? 1 : 0, b);
  }
}

int main() {
  char fmt[16] = {0};
  if (std::scanf("%15s", fmt) != 1) return 2;
  if (!std::strcmp(fmt, "bf16")) run<lsq::EncBF16>();
  else if (!std::strcmp(fmt, "bf16x3")) run_bf16x3();
  else if (!std::strcmp(fmt, "f16")) run<lsq::EncF16>();
  else if (!std::strcmp(fmt, "e4m3")) run<lsq::EncE4M3>();
  else if (!std::strcmp(fmt, "f32")) run<lsq::EncF32>();
  else if (!std::strcmp(fmt, "f32fast")) run_f32fast();
  else return 2;
  return 0;
}
