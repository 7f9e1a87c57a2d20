// Host harness for the tensor-core sketch planner (lsq::plan_sketch_tc and the
// deferred-correction list sizes) linked against the built library: reads lines
// "fmt s m ncols num_sms" and prints
// "ok bn nsub ngroups mtiles splits kchunk s_pad stages nt rowb smem rec_cap rec_lists".
// No CUDA call is made, so it runs without a GPU.
#include <cstdint>
#include <cstdio>

#include "kernels.h"

int main() {
  int fmt, sms;
  long long s, m, ncols;
  while (std::scanf("%d %lld %lld %lld %d", &fmt, &s, &m, &ncols, &sms) == 5) {
    lsq::SketchPlan p{};
    const bool ok = lsq::plan_sketch_tc(fmt, s, m, ncols, sms, &p);
    if (!ok) {
      std::printf("0\n");
      continue;
    }
    std::printf("1 %d %d %d %d %d %lld %lld %d %d %d %zu %u %lld\n", p.bn, p.nsub, p.ngroups, p.mtiles,
                p.splits, (long long)p.kchunk, (long long)p.s_pad, p.stages, p.nt, p.rowb, p.smem,
                lsq::sketch_rec_cap(p), (long long)lsq::sketch_rec_lists(p));
  }
  return 0;
}
