// Host harness for csrc/cast.cuh: reads "fmt" then lines "u_hex k" (FP64 bits
// and a power-of-two exponent) and prints "ok t0 t1 t2" (hex bit patterns) for
// the integer rounding of 2^k * x into fmt (bf16, f16, e4m3, f32, bf16x3).
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "cast.cuh"

template <class F, bool S3>
static void run() {
  unsigned long long u;
  int k;
  while (std::scanf("%llx %d", &u, &k) == 2) {
    uint32_t t[3];
    const bool ok = lsq::cast_terms_int<F, S3>((uint64_t)u, k, t);
    std::printf("%d %x %x %x\n", ok ? 1 : 0, t[0], t[1], t[2]);
  }
}

int main() {
  char fmt[16] = {0};
  if (std::scanf("%15s", fmt) != 1) return 2;
  if (!std::strcmp(fmt, "bf16")) run<lsq::EncBF16, false>();
  else if (!std::strcmp(fmt, "bf16x3")) run<lsq::EncBF16, true>();
  else if (!std::strcmp(fmt, "f16")) run<lsq::EncF16, false>();
  else if (!std::strcmp(fmt, "e4m3")) run<lsq::EncE4M3, false>();
  else if (!std::strcmp(fmt, "f32")) run<lsq::EncF32, false>();
  else return 2;
  return 0;
}
