// Batched solves: Algorithms 1 and 2 for a batch of problems of uneven m and n with
// every stage as one grouped launch over all problems (batch.h): the cast, the
// tensor-core sketch (one persistent-style grid over every problem's (tile, column
// group, split) items with per-problem tensor maps and Philox keys), the QR (one CTA per
// problem), LSQR and FGMRES (one pass launch per iteration covering every problem's
// rows, with per-problem done flags), all iteration batches replayed as CUDA graphs.
//
// Each problem is computed with the same blocking whatever the batch holds, so its
// result is that of the same problem in a batch of one.
#include <cmath>
#include <cstring>
#include <vector>

#include "batch.h"
#include "host.h"

namespace {

using namespace lsq;

constexpr size_t kAlign = 256;
constexpr int64_t kPassRowsPerCta = 1024;   // rows of A per CTA of a grouped pass
constexpr int64_t kArnRowsPerCta = 8192;    // rows of the (m + n) vectors per Arnoldi CTA

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Per-problem byte offsets into one workspace buffer.
struct Arena {
  std::vector<size_t> off;
  size_t total = 0;
  char* base = nullptr;
  template <typename T>
  T* at(size_t p) const {
    return reinterpret_cast<T*>(base + off[p]);
  }
};

Arena make_arena(lsq_handle* h, const char* name, const std::vector<size_t>& bytes, bool zero = false) {
  Arena a;
  a.off.resize(bytes.size());
  for (size_t p = 0; p < bytes.size(); ++p) {
    a.off[p] = a.total;
    a.total += align_up(bytes[p]);
  }
  a.base = static_cast<char*>(ws(h, name, a.total > 0 ? a.total : kAlign, zero));
  return a;
}

// Prefix sums of per-problem CTA counts (the `start` table of a grouped launch).
struct Groups {
  int* dev = nullptr;
  int64_t total = 0;
};

Groups make_groups(lsq_handle* h, const char* name, const std::vector<int64_t>& counts) {
  std::vector<int> start(counts.size() + 1, 0);
  int64_t t = 0;
  for (size_t p = 0; p < counts.size(); ++p) {
    start[p] = (int)t;
    t += counts[p];
  }
  start[counts.size()] = (int)t;
  if (t > 2147483647LL) throw StatusFail{LSQ_E_INVAL};
  Groups g;
  g.total = t;
  g.dev = static_cast<int*>(ws(h, name, start.size() * sizeof(int)));
  CK(cudaMemcpyAsync(g.dev, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  return g;
}

template <typename T>
T* upload(lsq_handle* h, const char* name, const std::vector<T>& v) {
  T* d = static_cast<T*>(ws(h, name, v.size() * sizeof(T) + 16));
  if (!v.empty())
    CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return d;
}

template <typename T>
std::vector<T> download(lsq_handle* h, const T* d, size_t count) {
  std::vector<T> v(count);
  if (count) {
    CK(cudaMemcpyAsync(v.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return v;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct BatchCtx {
  lsq_handle* h;
  cudaStream_t st;
  int np;
  const lsq_problem* probs;
  lsq_prec us, up, uw, ur;
  double tol;
  lsq_opts o;
  double alpha;
  std::vector<int64_t> m, n, s, lda, lda32;
  int64_t pass_grid = 0;   // CTAs of the persistent grouped passes (0: one per item)
};

// A graph of `body` cached under `key` (the pointers it captured are part of the key).
CachedGraph* batch_graph(BatchCtx& b, const std::string& key, const std::function<void()>& body) {
  Ctx c{};
  c.h = b.h;
  c.st = b.st;
  return get_graph(c, key, body);
}

void run_graph(BatchCtx& b, CachedGraph* G) {
  CK(cudaGraphLaunch(G->e, b.st));
  b.h->launches += G->kernels;
}

#define LB(...)             \
  do {                      \
    CK((__VA_ARGS__));      \
    ++b.h->launches;        \
  } while (0)

// The tile autotuner: the grid of the persistent grouped passes.  Candidates are one CTA
// per item and 32, 16, 8 or 4 CTAs per SM; each runs the given pass (whose outputs the
// solve overwrites) once to warm up and three times under CUDA events, and the fastest is
// kept for this batch shape in the handle.  Every candidate computes every item the same
// way, so the choice changes the speed only.
int64_t tune_pass_grid(BatchCtx& b, const PassArgs<float>* tab, const Groups& g, size_t smem) {
  if (b.o.batch_grid > 0) return b.o.batch_grid;
  std::string key = "pass";
  {
    uint64_t hsh = 1469598103934665603ull;
    for (int p = 0; p < b.np; ++p) {
      hsh = (hsh ^ (uint64_t)b.m[p]) * 1099511628211ull;
      hsh = (hsh ^ (uint64_t)b.lda32[p]) * 1099511628211ull;
    }
    key += ":" + std::to_string(b.np) + ":" + std::to_string(hsh);
  }
  auto it = b.h->tuned.find(key);
  if (it != b.h->tuned.end()) return it->second;
  std::vector<int64_t> cands = {0};
  for (int per : {32, 16, 8, 4}) {
    const int64_t gsz = (int64_t)per * b.h->num_sms;
    if (gsz < g.total) cands.push_back(gsz);
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int64_t best = 0;
  float best_ms = 0.f;
  for (const int64_t c : cands) {
    CK(launch_grouped_pass<float>(PM_LSQR, 4, 2, tab, g.dev, g.total, b.np, smem, b.st, c));
    CK(cudaEventRecord(e0, b.st));
    for (int r = 0; r < 3; ++r) CK(launch_grouped_pass<float>(PM_LSQR, 4, 2, tab, g.dev, g.total, b.np, smem, b.st, c));
    CK(cudaEventRecord(e1, b.st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    b.h->launches += 4;
    if (c == cands.front() || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b.h->tuned[key] = best;
  return best;
}

// The FGMRES solves of one refinement step for every active problem (Alg. 2, FGMRES
// solve), products in TOP; fills per-problem iteration counts, relative residuals,
// second passes and the four update norms.
template <typename TOP>
void batch_fgmres(BatchCtx& b, const std::vector<const TOP*>& Aop, const std::vector<int64_t>& ldop,
                  const std::vector<Tri<TOP>>& tri, const std::vector<double*>& f, const std::vector<double*>& hv,
                  const std::vector<double*>& x, const std::vector<double*>& r, int* skip_dev, int gmax,
                  double gtol, std::vector<GmState>& states, std::vector<double>& norms) {
  lsq_handle* h = b.h;
  const int np = b.np;
  const int maxc = gmax + 1, ldh = gmax + 1;
  const bool f32 = sizeof(TOP) == 4;
  std::vector<int64_t> pass_ctas(np), arn_ctas(np), col_ctas(np);
  std::vector<size_t> szV(np), szZ(np), szW(np), szAz(np), szV32(np), szP(np), szS(np), szH(np), szSmall(np),
      szDp(np), szNb(np), szP4(np);
  std::vector<int64_t> ldz(np);
  for (int p = 0; p < np; ++p) {
    const int64_t m = b.m[p], n = b.n[p], len = m + n;
    pass_ctas[p] = cdiv(m, kPassRowsPerCta);
    arn_ctas[p] = cdiv(len, kArnRowsPerCta);
    col_ctas[p] = cdiv(n, 32);
    ldz[p] = (n + 3) / 4 * 4 + 4;
    szV[p] = (size_t)len * maxc * 8;
    szZ[p] = (size_t)ldz[p] * maxc * sizeof(TOP);
    szW[p] = (size_t)len * 8;
    szAz[p] = (size_t)(m + 8) * sizeof(TOP);
    szV32[p] = f32 ? (size_t)(m + 8) * 4 : 16;
    szP[p] = (size_t)pass_ctas[p] * n * sizeof(TOP);
    szS[p] = (size_t)ldz[p] * sizeof(TOP);
    szH[p] = (size_t)ldh * gmax * 8;
    szSmall[p] = (size_t)(maxc + 4) * 8;
    szDp[p] = (size_t)(maxc + 2) * arn_ctas[p] * 8;
    szNb[p] = (size_t)arn_ctas[p] * 8;
    szP4[p] = (size_t)arn_ctas[p] * 4 * 8;
  }
  const char* tg = f32 ? "32" : "64";
  auto nm = [&](const char* base) {
    static thread_local std::string s;
    s = std::string("bgm_") + base + tg;
    return s.c_str();
  };
  Arena aV = make_arena(h, nm("V"), szV), aZ = make_arena(h, nm("Z"), szZ, true), aW = make_arena(h, nm("W"), szW);
  Arena aAz = make_arena(h, nm("Az"), szAz), aV32 = make_arena(h, nm("V32"), szV32), aP = make_arena(h, nm("P"), szP);
  Arena aS = make_arena(h, nm("S"), szS, true), aH = make_arena(h, nm("H"), szH, true);
  Arena aCs = make_arena(h, nm("cs"), szSmall), aSn = make_arena(h, nm("sn"), szSmall),
        aG = make_arena(h, nm("g"), szSmall, true), aY = make_arena(h, nm("y"), szSmall),
        aH1 = make_arena(h, nm("h1"), szSmall), aH2 = make_arena(h, nm("h2"), szSmall);
  Arena aDp = make_arena(h, nm("Dp"), szDp), aSq = make_arena(h, nm("sq"), szNb), aP4 = make_arena(h, nm("p4"), szP4);
  // states and norms of all problems in one array each (one copy reads them all)
  GmState* sts = static_cast<GmState*>(ws(h, nm("st"), (size_t)np * sizeof(GmState)));
  double* nrms = static_cast<double*>(ws(h, nm("nrm"), (size_t)np * 32));
  Groups gPass = make_groups(h, nm("gpass"), pass_ctas), gArn = make_groups(h, nm("garn"), arn_ctas),
         gCol = make_groups(h, nm("gcol"), col_ctas);
  // tables
  std::vector<GTrsv<TOP, double, TOP>> tz(np);
  std::vector<PassArgs<TOP>> tp(np);
  std::vector<GColsum<TOP, TOP>> tc(np);
  std::vector<GTrsv<TOP, TOP, double>> tw(np);
  std::vector<GGm> tg_(np);
  std::vector<GmState> init(np);
  for (int p = 0; p < np; ++p) {
    const int64_t m = b.m[p], n = b.n[p], ld = m + n;
    GmState* st = sts + p;
    double* V = aV.at<double>(p);
    TOP* Zb = aZ.at<TOP>(p);
    double* wv = aW.at<double>(p);
    TOP* az = aAz.at<TOP>(p);
    float* v32 = f32 ? aV32.at<float>(p) : nullptr;
    TOP* P = aP.at<TOP>(p);
    TOP* sb = aS.at<TOP>(p);
    const int* dn = &st->done;
    const int* jp = &st->j;
    tz[p] = GTrsv<TOP, double, TOP>{tri[p].R, tri[p].DU, tri[p].ld, (int)n, V + m, 1.0, Zb, dn, jp, ld, ldz[p]};
    PassArgs<TOP> q{};
    q.A = Aop[p];
    q.lda = ldop[p];
    q.m = m;
    q.n = (int)n;
    q.nv = f32 ? (int)(ldop[p] / 4) : (int)n;
    q.x = Zb;
    q.xstr = ldz[p];
    q.jp = jp;
    if (f32) {
      q.v = reinterpret_cast<const TOP*>(v32);
      q.vstr = 0;
    } else {
      q.v = reinterpret_cast<const TOP*>(V);
      q.vstr = ld;
    }
    q.az = az;
    q.Pblk = P;
    q.done = dn;
    tp[p] = q;
    tc[p] = GColsum<TOP, TOP>{P, (int)pass_ctas[p], n, nullptr, 1.0, sb, dn};
    tw[p] = GTrsv<TOP, TOP, double>{tri[p].L, tri[p].DL, tri[p].ld, (int)n, sb, 1.0, wv + m, dn, nullptr, 0, 0};
    GGm g{};
    g.V = V;
    g.ld = ld;
    g.m = m;
    g.n = n;
    g.w = wv;
    g.az = az;
    g.az_f32 = f32 ? 1 : 0;
    g.st = st;
    g.maxc = maxc;
    g.ldh = ldh;
    g.Dp = aDp.at<double>(p);
    g.hs1 = aH1.at<double>(p);
    g.hs2 = aH2.at<double>(p);
    g.H = aH.at<double>(p);
    g.cs = aCs.at<double>(p);
    g.sn = aSn.at<double>(p);
    g.g = aG.at<double>(p);
    g.y = aY.at<double>(p);
    g.v32 = v32;
    g.alpha = b.alpha;
    g.f = f[p];
    g.h = hv[p];
    g.sqp = aSq.at<double>(p);
    g.skip = skip_dev + p;
    g.Zb = Zb;
    g.zb_f32 = f32 ? 1 : 0;
    g.ldz = ldz[p];
    g.r = r[p];
    g.x = x[p];
    g.p4 = aP4.at<double>(p);
    g.nrm = nrms + 4 * p;
    tg_[p] = g;
    GmState s0{};
    s0.tol = gtol;
    s0.maxit = gmax;
    init[p] = s0;
  }
  auto* dz = upload(h, nm("tz"), tz);
  auto* dp = upload(h, nm("tp"), tp);
  auto* dc = upload(h, nm("tc"), tc);
  auto* dw = upload(h, nm("tw"), tw);
  auto* dg = upload(h, nm("tg"), tg_);
  CK(cudaMemcpyAsync(sts, init.data(), (size_t)np * sizeof(GmState), cudaMemcpyHostToDevice, b.st));
  LB(launch_grouped_gm_init(dg, gArn.dev, gArn.total, np, b.st));
  const int vw = f32 ? 4 : 1, vpl = f32 ? 2 : 8;
  int64_t maxw = 0;
  for (int p = 0; p < np; ++p) maxw = std::max<int64_t>(maxw, f32 ? ldop[p] : b.n[p]);
  const size_t pass_smem = (size_t)8 * maxw * sizeof(TOP);
  auto body = [&]() {
    for (int k = 0; k < kBatch; ++k) {
      LB(launch_grouped_trsv<TOP, double, TOP>(true, dz, np, b.st));
      LB(launch_grouped_pass<TOP>(PM_FGM, vw, vpl, dp, gPass.dev, gPass.total, np, pass_smem, b.st, b.pass_grid));
      LB(launch_grouped_colsum<TOP, TOP>(dc, gCol.dev, gCol.total, np, b.st));
      LB(launch_grouped_trsv<TOP, TOP, double>(false, dw, np, b.st));
      LB(launch_grouped_arnoldi(dg, gArn.dev, gArn.total, np, b.st));
      b.h->launches += 6;
    }
  };
  CachedGraph* G = b.o.no_graph ? nullptr
                                : batch_graph(b, graph_key(f32 ? "bfgm32" : "bfgm64",
                                                           {PV(dz), PV(dp), PV(dc), PV(dw), PV(dg), PV(gPass.dev),
                                                            gPass.total, PV(gArn.dev), gArn.total, np,
                                                            (int64_t)pass_smem, b.pass_grid}),
                                              body);
  states.assign(np, GmState{});
  for (int it = 0; it <= gmax + kBatch; it += kBatch) {
    if (G) run_graph(b, G);
    else body();
    // all problems done?
    bool all = true;
    CK(cudaMemcpyAsync(states.data(), sts, (size_t)np * sizeof(GmState), cudaMemcpyDeviceToHost, b.st));
    CK(cudaStreamSynchronize(b.st));
    for (int p = 0; p < np; ++p) all = all && states[p].done;
    if (all) break;
  }
  check_dev_error(h);
  LB(launch_grouped_gm_update(dg, gArn.dev, gArn.total, np, b.st));
  b.h->launches += 2;
  norms.assign((size_t)np * 4, 0.0);
  CK(cudaMemcpyAsync(norms.data(), nrms, (size_t)np * 32, cudaMemcpyDeviceToHost, b.st));
  CK(cudaStreamSynchronize(b.st));
}

}  // namespace

lsq_status lsq_batch_grouped(lsq_handle* h, int32_t nprob, const lsq_problem* probs, lsq_prec u_s, lsq_prec u_p,
                             lsq_prec u_w, lsq_prec u_r, double tol, const lsq_opts* opts, int32_t* statuses,
                             lsq_info* infos) {
  BatchCtx b{};
  b.h = h;
  b.st = h->stream;
  b.np = nprob;
  b.probs = probs;
  b.us = u_s;
  b.up = u_p;
  b.uw = u_w;
  b.ur = u_r;
  b.tol = tol;
  if (opts) b.o = *opts;
  else std::memset(&b.o, 0, sizeof(b.o));
  b.alpha = b.o.aug_alpha > 0.0 ? b.o.aug_alpha : 1.0;
  const int fmt = fmt_of(u_s);
  const bool tc = fmt == FMT_F16 || fmt == FMT_BF16 || fmt == FMT_E4M3 || fmt == FMT_BF16X3;
  if (!tc || u_w != LSQ_F32 || u_r != LSQ_F64 || (u_p != LSQ_F32 && u_p != LSQ_F64) || b.o.sketch_kind != 0 ||
      b.o.Y_in || b.o.R_in || b.o.ops_escalated || b.o.timing)
    return LSQ_E_UNSUPPORTED;
  const int np = nprob;
  b.m.resize(np);
  b.n.resize(np);
  b.s.resize(np);
  b.lda.resize(np);
  b.lda32.resize(np);
  std::vector<SketchPlan> plans(np);
  for (int p = 0; p < np; ++p) {
    b.m[p] = probs[p].m;
    b.n[p] = probs[p].n;
    b.s[p] = probs[p].s;
    b.lda[p] = probs[p].lda > 0 ? probs[p].lda : probs[p].n;
    b.lda32[p] = (b.n[p] + 3) / 4 * 4;
    if (b.n[p] > 256 || b.s[p] > 1024 || !probs[p].x) return LSQ_E_UNSUPPORTED;
  }
  // one kernel instantiation for the batch: the smallest stage count of the plans and the
  // largest shared-memory size (a plan's layout needs at most its own stage count)
  int stages = 4;
  size_t sk_smem = 0;
  for (int p = 0; p < np; ++p) {
    // the plan depends on the problem alone (about one CTA-wave share per 8192 rows), so
    // that its result does not depend on the rest of the batch
    const int share = (int)std::min<int64_t>(h->num_sms, std::max<int64_t>(1, b.m[p] / 8192));
    if (!plan_sketch_tc(fmt, b.s[p], b.m[p], b.n[p] + 1, share, &plans[p], b.o.sketch_kchunk))
      return LSQ_E_UNSUPPORTED;
    if (plans[p].splits > 65535) return LSQ_E_UNSUPPORTED;
    stages = std::min(stages, plans[p].stages);
    sk_smem = std::max(sk_smem, plans[p].smem);
  }
  std::vector<lsq_info> local((size_t)np);
  lsq_info* inf = infos ? infos : local.data();
  for (int p = 0; p < np; ++p) std::memset(&inf[p], 0, sizeof(lsq_info));

  return run_guarded(h, nullptr, [&]() -> lsq_status {
    StageTimer ttot(h, ST_TOTAL);
    // ------------------------------------------------------------ cast (a1)
    std::vector<size_t> szC(np), szA32(np), szK(np), szBt(np), szPart(np), szY(np);
    std::vector<int64_t> cmx(np), exps(np), castc(np), skc(np), redc(np);
    for (int p = 0; p < np; ++p) {
      const SketchPlan& pl = plans[p];
      const int64_t rows = (int64_t)pl.ngroups * pl.bn;
      szC[p] = (size_t)(b.n[p] + 1) * 8;
      szA32[p] = (size_t)b.m[p] * b.lda32[p] * 4;
      szK[p] = (size_t)(b.n[p] + 1) * 4;
      szBt[p] = bt_bytes(fmt, b.m[p], rows);
      szPart[p] = (size_t)pl.splits * pl.ncols * pl.s_pad * 4;
      szY[p] = (size_t)b.s[p] * (b.n[p] + 1) * 8;
      cmx[p] = cdiv(b.m[p], kGroupedColmaxRows);
      exps[p] = cdiv(b.n[p] + 1, 256);
      castc[p] = cast_row_tiles(fmt, b.m[p]) * cdiv(rows, 32);
      skc[p] = (int64_t)pl.mtiles * pl.ngroups * pl.splits;
      redc[p] = cdiv(b.s[p], 256) * (b.n[p] + 1);
    }
    Arena aC = make_arena(h, "b_cmax", szC, true), aA32 = make_arena(h, "b_a32", szA32),
          aK = make_arena(h, "b_kexp", szK), aBt = make_arena(h, "b_bt", szBt),
          aPart = make_arena(h, "b_part", szPart), aY = make_arena(h, "b_Y", szY);
    std::vector<GCast> tcast(np);
    for (int p = 0; p < np; ++p) {
      const SketchPlan& pl = plans[p];
      GCast g{};
      g.A = probs[p].A;
      g.lda = b.lda[p];
      g.b = probs[p].b;
      g.m = b.m[p];
      g.n = b.n[p];
      g.cmax = aC.at<unsigned long long>(p);
      g.a32 = aA32.at<float>(p);
      g.lda32 = b.lda32[p];
      g.kexp = aK.at<int>(p);
      g.Bt = aBt.at<void>(p);
      g.plane_rows = (int64_t)pl.ngroups * pl.bn;
      g.cast_gx = cast_row_tiles(fmt, b.m[p]);
      tcast[p] = g;
    }
    {
      StageTimer t(h, ST_CAST);
      GCast* dcast = upload(h, "b_tcast", tcast);
      Groups gc = make_groups(h, "b_gcmax", cmx), ge = make_groups(h, "b_gexp", exps),
             gk = make_groups(h, "b_gcast", castc);
      const int tsc = b.o.no_colscale ? -1 : (fmt == FMT_E4M3 ? 7 : 14);
      LB(launch_grouped_cast(fmt, dcast, gc.dev, gc.total, ge.dev, ge.total, gk.dev, gk.total, np, tsc, h->d_err,
                             b.st));
      b.h->launches += 2;
    }
    check_dev_error(h);   // a NaN or an infinity in some A or b
    // ------------------------------------------------------------ sketch (a2, a3)
    {
      StageTimer t(h, ST_SKETCH);
      std::vector<SketchTcArgs> targs(np);
      std::vector<CUtensorMap> maps(np);
      std::vector<GReduce> tred(np);
      for (int p = 0; p < np; ++p) {
        const SketchPlan& pl = plans[p];
        const int64_t rows = (int64_t)pl.ngroups * pl.bn;
        if (!encode_bt_tmap(&maps[p], aBt.at<void>(p), fmt, (int64_t)pl.nt * rows, b.m[p], pl.bn / pl.nsub, pl.rowb))
          throw StatusFail{LSQ_E_UNSUPPORTED};
        targs[p] = sketch_tc_args(pl, probs[p].seed, aPart.at<float>(p), h->d_err);
        tred[p] = GReduce{aPart.at<float>(p), pl.splits, pl.ncols, b.s[p], pl.s_pad, aK.at<int>(p), aY.at<double>(p)};
      }
      SketchGroup sg{};
      sg.tab = upload(h, "b_targs", targs);
      sg.maps = upload(h, "b_maps", maps);
      Groups gs = make_groups(h, "b_gsk", skc);
      sg.start = gs.dev;
      sg.nprob = np;
      CK(cudaStreamSynchronize(b.st));
      LB(launch_sketch_tc_grouped(fmt, stages, sg, gs.total, sk_smem, b.st));
      Groups gr = make_groups(h, "b_gred", redc);
      GReduce* dred = upload(h, "b_tred", tred);
      LB(launch_grouped_sketch_reduce(dred, gr.dev, gr.total, np, b.st));
      CK(cudaStreamSynchronize(b.st));
    }
    check_dev_error(h);
    // ------------------------------------------------------------ QR (a4), R copies, x_s
    std::vector<size_t> szW(np), szN(np), szNN(np), szR32(np), szR64(np), szD32(np), szD64(np);
    std::vector<int64_t> ncol(np), nblk32(np);
    const bool qr64 = u_p == LSQ_F64;
    for (int p = 0; p < np; ++p) {
      const int64_t n = b.n[p], ld32 = tri_ld(n, 4), ld64 = tri_ld(n, 8);
      szW[p] = (size_t)b.s[p] * (n + 1) * (qr64 ? 8 : 4);
      szN[p] = (size_t)(n + 4) * 8;
      szNN[p] = (size_t)n * n * 8;
      szR32[p] = (size_t)ld32 * n * 4;
      szR64[p] = (size_t)ld64 * n * 8;
      szD32[p] = (size_t)cdiv(n, 32) * 1024 * 4;
      szD64[p] = (size_t)cdiv(n, 32) * 1024 * 8;
      ncol[p] = n;
      nblk32[p] = cdiv(n, 32);
    }
    Arena aW = make_arena(h, "b_qrw", szW), aDg = make_arena(h, "b_diag", szN), aR = make_arena(h, "b_R", szNN),
          aCv = make_arena(h, "b_c", szN), aR32 = make_arena(h, "b_R32", szR32), aL32 = make_arena(h, "b_L32", szR32),
          aDU32 = make_arena(h, "b_DU32", szD32), aDL32 = make_arena(h, "b_DL32", szD32),
          aR64 = make_arena(h, "b_R64", szR64), aL64 = make_arena(h, "b_L64", szR64),
          aDU64 = make_arena(h, "b_DU64", szD64), aDL64 = make_arena(h, "b_DL64", szD64),
          aX0 = make_arena(h, "b_x0", szN);
    double* kapd = static_cast<double*>(ws(h, "b_kap", (size_t)np * 8));
    Groups gcol = make_groups(h, "b_gqrcol", ncol), gblk = make_groups(h, "b_gqrblk", nblk32);
    std::vector<Tri<float>> tri32(np);
    std::vector<Tri<double>> tri64(np);
    {
      StageTimer t(h, ST_QR);
      std::vector<GPrepR> tprep(np);
      for (int p = 0; p < np; ++p) {
        const int64_t n = b.n[p];
        tri32[p] = Tri<float>{aR32.at<float>(p), aL32.at<float>(p), aDU32.at<float>(p), aDL32.at<float>(p), n,
                              tri_ld(n, 4), h->d_err};
        tri64[p] = Tri<double>{aR64.at<double>(p), aL64.at<double>(p), aDU64.at<double>(p), aDL64.at<double>(p), n,
                               tri_ld(n, 8), h->d_err};
        tprep[p] = GPrepR{aR.at<double>(p), n, tri32[p], tri64[p], kapd + p};
      }
      if (qr64) {
        std::vector<GQr<double>> tq(np);
        for (int p = 0; p < np; ++p)
          tq[p] = GQr<double>{aY.at<double>(p), aW.at<double>(p), b.s[p], b.n[p], aDg.at<double>(p), aR.at<double>(p),
                              aCv.at<double>(p)};
        LB(launch_grouped_qr<double>(upload(h, "b_tq", tq), gcol.dev, gcol.total, np, 256, b.st));
      } else {
        std::vector<GQr<float>> tq(np);
        for (int p = 0; p < np; ++p)
          tq[p] = GQr<float>{aY.at<double>(p), aW.at<float>(p), b.s[p], b.n[p], aDg.at<double>(p), aR.at<double>(p),
                             aCv.at<double>(p)};
        LB(launch_grouped_qr<float>(upload(h, "b_tq", tq), gcol.dev, gcol.total, np, 256, b.st));
      }
      LB(launch_grouped_prepare_r(upload(h, "b_tprep", tprep), gcol.dev, gcol.total, gblk.dev, gblk.total, np,
                                  b.st));
      b.h->launches += 4;
      if (qr64) {
        std::vector<GTrsv<double, double, double>> tx(np);
        for (int p = 0; p < np; ++p)
          tx[p] = GTrsv<double, double, double>{tri64[p].R, tri64[p].DU, tri64[p].ld, (int)b.n[p], aCv.at<double>(p),
                                                1.0, aX0.at<double>(p), nullptr, nullptr, 0, 0};
        LB(launch_grouped_trsv<double, double, double>(true, upload(h, "b_txs", tx), np, b.st));
      } else {
        std::vector<GTrsv<float, double, double>> tx(np);
        for (int p = 0; p < np; ++p)
          tx[p] = GTrsv<float, double, double>{tri32[p].R, tri32[p].DU, tri32[p].ld, (int)b.n[p], aCv.at<double>(p),
                                               1.0, aX0.at<double>(p), nullptr, nullptr, 0, 0};
        LB(launch_grouped_trsv<float, double, double>(true, upload(h, "b_txs", tx), np, b.st));
      }
      CK(cudaStreamSynchronize(b.st));
    }
    std::vector<double> kap = download(h, kapd, (size_t)np);
    std::vector<int> failed(np, 0);
    for (int p = 0; p < np; ++p) {
      inf[p].kappa_R_est = kap[p];
      inf[p].us_used = (int32_t)u_s;
      inf[p].sketches = 1;
      inf[p].aug_alpha = b.alpha;
      if (!(kap[p] < INFINITY)) failed[p] = 1;
      else if (kap[p] * unit_roundoff(u_s) >= 1.0) inf[p].flags |= LSQ_WARN_COND;
    }
    // ------------------------------------------------------------ LSQR (a5, a6)
    std::vector<int64_t> pcta(np), ncta(np), mcta(np);
    std::vector<size_t> szU(np), szVec(np), szPb(np), szSq(np), szM8(np), szM4(np);
    for (int p = 0; p < np; ++p) {
      pcta[p] = cdiv(b.m[p], kPassRowsPerCta);
      ncta[p] = cdiv(b.n[p], 32);
      mcta[p] = cdiv(b.m[p], 256);
      szU[p] = (size_t)(b.m[p] + 8) * 4;
      szVec[p] = (size_t)(b.lda32[p] + 8) * 4;
      szPb[p] = (size_t)pcta[p] * b.n[p] * 4;
      szSq[p] = (size_t)pcta[p] * 8;
      szM8[p] = (size_t)(b.m[p] + 8) * 8;
      szM4[p] = (size_t)(b.m[p] + 8) * 4;
    }
    Arena aU = make_arena(h, "b_u", szU), aB32 = make_arena(h, "b_b32", szM4), aT = make_arena(h, "b_t", szVec, true),
          aSv = make_arena(h, "b_sv", szVec, true), aVv = make_arena(h, "b_v", szVec, true),
          aWv = make_arena(h, "b_w", szVec, true), aZv = make_arena(h, "b_z", szVec, true),
          aPb = make_arena(h, "b_pb", szPb), aSqv = make_arena(h, "b_sq", szSq), aXl = make_arena(h, "b_xl", szN),
          aR0 = make_arena(h, "b_r0", szM8);
    LsqrState* lsd = static_cast<LsqrState*>(ws(h, "b_ls", (size_t)np * sizeof(LsqrState)));
    Groups gp = make_groups(h, "b_gpass", pcta), gn = make_groups(h, "b_gn", ncta), gm = make_groups(h, "b_gm", mcta);
    std::vector<LsqrState> lst(np);
    {
      StageTimer t(h, ST_LSQR);
      std::vector<GAxpby<double, double, float>> tb32(np), tneg(np);
      std::vector<GNorm> tnb(np);
      std::vector<PassArgs<float>> tp0(np), tp1(np);
      std::vector<GLsqrColsum<float>> tcs(np);
      std::vector<GLsqrStep<float>> tstep(np);
      std::vector<LsqrState> init(np);
      for (int p = 0; p < np; ++p) {
        LsqrState* ls = lsd + p;
        std::memset(&init[p], 0, sizeof(LsqrState));
        init[p].tol = tol;
        init[p].maxit = b.o.lsqr_maxit > 0 ? b.o.lsqr_maxit : (int)(2 * b.n[p]);
        if (failed[p]) {
          init[p].done = 1;
          init[p].maxit = 0;
        }
        tb32[p] = GAxpby<double, double, float>{probs[p].b, 1.0, nullptr, 0.0, aB32.at<float>(p), b.m[p], nullptr};
        tneg[p] = GAxpby<double, double, float>{aX0.at<double>(p), -1.0, nullptr, 0.0, aT.at<float>(p), b.n[p], nullptr};
        tnb[p] = GNorm{probs[p].b, b.m[p], &ls->normb};
        PassArgs<float> q{};
        q.A = aA32.at<float>(p);
        q.lda = b.lda32[p];
        q.m = b.m[p];
        q.n = (int)b.n[p];
        q.nv = (int)(b.lda32[p] / 4);
        q.x = aT.at<float>(p);
        q.uin = aB32.at<float>(p);
        q.uout = aU.at<float>(p);
        q.cu_ptr = nullptr;
        q.cu_mul = 1.0;
        q.Pblk = aPb.at<float>(p);
        q.sq = aSqv.at<double>(p);
        q.done = failed[p] ? &ls->done : nullptr;
        tp0[p] = q;
        q.uin = aU.at<float>(p);
        q.cu_ptr = &ls->cu;
        q.done = &ls->done;
        tp1[p] = q;
        tcs[p] = GLsqrColsum<float>{aPb.at<float>(p), (int)pcta[p], b.n[p], aSqv.at<double>(p), ls, aSv.at<float>(p)};
        tstep[p] = GLsqrStep<float>{tri32[p], aSv.at<float>(p), aVv.at<float>(p), aWv.at<float>(p), aZv.at<float>(p),
                                    aT.at<float>(p), ls};
      }
      CK(cudaMemcpyAsync(lsd, init.data(), (size_t)np * sizeof(LsqrState), cudaMemcpyHostToDevice, b.st));
      auto* db32 = upload(h, "b_tb32", tb32);
      auto* dneg = upload(h, "b_tneg", tneg);
      auto* dnb = upload(h, "b_tnb", tnb);
      auto* dp0 = upload(h, "b_tp0", tp0);
      auto* dp1 = upload(h, "b_tp1", tp1);
      auto* dcs = upload(h, "b_tcs", tcs);
      auto* dstep = upload(h, "b_tstep", tstep);
      CK(cudaStreamSynchronize(b.st));
      int64_t maxw = 0;
      for (int p = 0; p < np; ++p) maxw = std::max(maxw, b.lda32[p]);
      const size_t pass_smem = (size_t)8 * maxw * 4;
      LB(launch_grouped_axpby(db32, gm.dev, gm.total, np, b.st));
      LB(launch_grouped_norm(dnb, np, b.st));
      LB(launch_grouped_axpby(dneg, gn.dev, gn.total, np, b.st));
      // the persistent passes' grid: forced, cached for this batch shape, or chosen now by
      // timing this (repeatable) first pass with each candidate
      b.pass_grid = tune_pass_grid(b, dp0, gp, pass_smem);
      LB(launch_grouped_pass<float>(PM_LSQR, 4, 2, dp0, gp.dev, gp.total, np, pass_smem, b.st, b.pass_grid));
      LB(launch_grouped_lsqr_colsum<float>(dcs, gn.dev, gn.total, np, true, b.st));
      LB(launch_grouped_lsqr_step<float>(dstep, np, true, b.st));
      auto body = [&]() {
        for (int k = 0; k < kBatch; ++k) {
          LB(launch_grouped_pass<float>(PM_LSQR, 4, 2, dp1, gp.dev, gp.total, np, pass_smem, b.st, b.pass_grid));
          LB(launch_grouped_lsqr_colsum<float>(dcs, gn.dev, gn.total, np, false, b.st));
          LB(launch_grouped_lsqr_step<float>(dstep, np, false, b.st));
        }
      };
      CachedGraph* G = b.o.no_graph ? nullptr
                                    : batch_graph(b, graph_key("blsqr", {PV(dp1), PV(dcs), PV(dstep), PV(gp.dev),
                                                                         gp.total, np, (int64_t)pass_smem,
                                                                         b.pass_grid}),
                                                  body);
      int maxit_all = 0;
      for (int p = 0; p < np; ++p) maxit_all = std::max(maxit_all, init[p].maxit);
      for (int it = 0; it <= maxit_all + kBatch; it += kBatch) {
        if (G) run_graph(b, G);
        else body();
        CK(cudaMemcpyAsync(lst.data(), lsd, (size_t)np * sizeof(LsqrState), cudaMemcpyDeviceToHost, b.st));
        CK(cudaStreamSynchronize(b.st));
        bool all = true;
        for (int p = 0; p < np; ++p) all = all && lst[p].done;
        if (all) break;
      }
      // x_0 = x_s + R^-1 z
      std::vector<GTrsv<float, float, float>> tz(np);
      std::vector<GAxpby<float, double, double>> tx(np);
      for (int p = 0; p < np; ++p) {
        tz[p] = GTrsv<float, float, float>{tri32[p].R, tri32[p].DU, tri32[p].ld, (int)b.n[p], aZv.at<float>(p), 1.0,
                                           aT.at<float>(p), nullptr, nullptr, 0, 0};
        tx[p] = GAxpby<float, double, double>{aT.at<float>(p), 1.0, aX0.at<double>(p), 1.0, aXl.at<double>(p), b.n[p],
                                              nullptr};
      }
      LB(launch_grouped_trsv<float, float, float>(true, upload(h, "b_ttz", tz), np, b.st));
      LB(launch_grouped_axpby(upload(h, "b_ttx", tx), gn.dev, gn.total, np, b.st));
      CK(cudaStreamSynchronize(b.st));
    }
    for (int p = 0; p < np; ++p) {
      inf[p].lsqr_its = lst[p].its;
      inf[p].lsqr_flag = lst[p].flag;
      inf[p].lsqr_normr = lst[p].normr;
      inf[p].lsqr_normar = lst[p].normar;
      inf[p].lsqr_normA = lst[p].normA;
    }
    // ------------------------------------------------------------ r_0 = b - A x_0 (u), x, r
    {
      StageTimer t(h, ST_RES);
      std::vector<GAxpby<double, double, float>> tneg(np);
      std::vector<PassArgs<float>> tq(np);
      std::vector<GAxpby<float, double, double>> tr(np);
      for (int p = 0; p < np; ++p) {
        tneg[p] = GAxpby<double, double, float>{aXl.at<double>(p), -1.0, nullptr, 0.0, aT.at<float>(p), b.n[p], nullptr};
        PassArgs<float> q{};
        q.A = aA32.at<float>(p);
        q.lda = b.lda32[p];
        q.m = b.m[p];
        q.n = (int)b.n[p];
        q.nv = (int)(b.lda32[p] / 4);
        q.x = aT.at<float>(p);
        q.uin = aB32.at<float>(p);
        q.uout = aU.at<float>(p);
        q.cu_mul = 1.0;
        q.Pblk = aPb.at<float>(p);
        q.sq = aSqv.at<double>(p);
        tq[p] = q;
        tr[p] = GAxpby<float, double, double>{aU.at<float>(p), 1.0, nullptr, 0.0, aR0.at<double>(p), b.m[p], nullptr};
      }
      int64_t maxw = 0;
      for (int p = 0; p < np; ++p) maxw = std::max(maxw, b.lda32[p]);
      LB(launch_grouped_axpby(upload(h, "b_tn2", tneg), gn.dev, gn.total, np, b.st));
      LB(launch_grouped_pass<float>(PM_LSQR, 4, 2, upload(h, "b_tq2", tq), gp.dev, gp.total, np, (size_t)8 * maxw * 4,
                                    b.st, b.pass_grid));
      LB(launch_grouped_axpby(upload(h, "b_tr2", tr), gm.dev, gm.total, np, b.st));
      CK(cudaStreamSynchronize(b.st));
    }
    // ------------------------------------------------------------ refinement (a7 - a9)
    std::vector<double*> xv(np), rv(np), fv(np), gv(np), hv(np);
    std::vector<size_t> szF(np), szG(np), szP64(np), szSkip(np, 4);
    for (int p = 0; p < np; ++p) {
      szF[p] = (size_t)(b.m[p] + 8) * 8;
      szG[p] = (size_t)(b.n[p] + 8) * 8;
      szP64[p] = (size_t)pcta[p] * b.n[p] * 8;
    }
    Arena aF = make_arena(h, "b_f", szF), aG = make_arena(h, "b_g", szG), aHv = make_arena(h, "b_h", szG),
          aP64 = make_arena(h, "b_p64", szP64), aSkip = make_arena(h, "b_skip", szSkip);
    int* skip_dev = static_cast<int*>(ws(h, "b_skipv", (size_t)np * 4 + 16));
    for (int p = 0; p < np; ++p) {
      xv[p] = probs[p].x;
      rv[p] = probs[p].r;
      fv[p] = aF.at<double>(p);
      gv[p] = aG.at<double>(p);
      hv[p] = aHv.at<double>(p);
    }
    // r may be NULL for a problem: it then lives in a workspace copy
    std::vector<size_t> szRw(np);
    for (int p = 0; p < np; ++p) szRw[p] = probs[p].r ? 16 : (size_t)(b.m[p] + 8) * 8;
    Arena aRw = make_arena(h, "b_rw", szRw);
    for (int p = 0; p < np; ++p)
      if (!probs[p].r) rv[p] = aRw.at<double>(p);
    auto restart = [&](const std::vector<int>& which) {
      for (int p = 0; p < np; ++p) {
        if (!which[p]) continue;
        CK(cudaMemcpyAsync(xv[p], aXl.at<double>(p), b.n[p] * 8, cudaMemcpyDeviceToDevice, b.st));
        CK(cudaMemcpyAsync(rv[p], aR0.at<double>(p), b.m[p] * 8, cudaMemcpyDeviceToDevice, b.st));
      }
    };
    std::vector<int> all1(np, 1);
    restart(all1);
    // residual tables (FP64 A; skipped problems take no residual)
    std::vector<PassArgs<double>> tres(np);
    std::vector<GColsum<double, double>> tcg(np);
    std::vector<GTrsv<double, double, double>> th(np);
    for (int p = 0; p < np; ++p) {
      PassArgs<double> q{};
      q.A = probs[p].A;
      q.lda = b.lda[p];
      q.m = b.m[p];
      q.n = (int)b.n[p];
      q.nv = (int)b.n[p];
      q.x = xv[p];
      q.r = rv[p];
      q.b = probs[p].b;
      q.f = fv[p];
      q.Pblk = aP64.at<double>(p);
      q.done = skip_dev + p;
      tres[p] = q;
      tcg[p] = GColsum<double, double>{aP64.at<double>(p), (int)pcta[p], b.n[p], nullptr, 1.0, gv[p], skip_dev + p};
      th[p] = GTrsv<double, double, double>{tri64[p].L, tri64[p].DL, tri64[p].ld, (int)b.n[p], gv[p], 1.0, hv[p],
                                            skip_dev + p, nullptr, 0, 0};
    }
    auto* dres = upload(h, "b_tres", tres);
    auto* dcg = upload(h, "b_tcg", tcg);
    auto* dth = upload(h, "b_th", th);
    int64_t maxn = 0;
    for (int p = 0; p < np; ++p) maxn = std::max(maxn, b.n[p]);
    const double u = unit_roundoff(u_w);
    const int irmax = b.o.ir_maxit > 0 ? b.o.ir_maxit : 30;
    const int gmax = std::min(b.o.gmres_maxit > 0 ? b.o.gmres_maxit : 50, kMaxGmresBatch);
    const double gtol = b.o.gmres_tol > 0 ? b.o.gmres_tol : tol;
    // FP32 products: the FP32 copy (rows padded to lda32); FP64 products (the Sec. 5 re-run): A itself
    std::vector<const float*> A32(np);
    std::vector<const double*> A64(np);
    std::vector<int64_t> ld32(np), ld64(np);
    for (int p = 0; p < np; ++p) {
      A32[p] = aA32.at<float>(p);
      ld32[p] = b.lda32[p];
      A64[p] = probs[p].A;
      ld64[p] = b.lda[p];
    }
    auto refine = [&](bool f64ops, std::vector<int>& active, std::vector<int>& conv) {
      std::vector<double> prev_dx(np, 0.0), prev_dr(np, 0.0);
      std::vector<int> skip(np);
      for (int p = 0; p < np; ++p) {
        inf[p].ir_its = 0;
        inf[p].gmres_its_total = 0;
        conv[p] = 0;
      }
      for (int i = 0; i < irmax; ++i) {
        bool any = false;
        for (int p = 0; p < np; ++p) {
          skip[p] = (active[p] && !conv[p]) ? 0 : 1;
          any = any || !skip[p];
        }
        if (!any) break;
        CK(cudaMemcpyAsync(skip_dev, skip.data(), (size_t)np * 4, cudaMemcpyHostToDevice, b.st));
        {
          StageTimer t(h, ST_RES);
          LB(launch_grouped_pass<double>(PM_RES, 1, 8, dres, gp.dev, gp.total, np, (size_t)8 * maxn * 8, b.st,
                                         b.pass_grid));
          LB(launch_grouped_colsum<double, double>(dcg, gn.dev, gn.total, np, b.st));
          LB(launch_grouped_trsv<double, double, double>(false, dth, np, b.st));
        }
        std::vector<GmState> gs;
        std::vector<double> nr;
        {
          StageTimer t(h, ST_FGMRES);
          if (f64ops) {
            batch_fgmres<double>(b, A64, ld64, tri64, fv, hv, xv, rv, skip_dev, gmax, gtol, gs, nr);
          } else {
            batch_fgmres<float>(b, A32, ld32, tri32, fv, hv, xv, rv, skip_dev, gmax, gtol, gs, nr);
          }
        }
        for (int p = 0; p < np; ++p) {
          if (skip[p]) continue;
          const double dr = std::sqrt(nr[(size_t)p * 4 + 0]), r2 = std::sqrt(nr[(size_t)p * 4 + 1]);
          const double dx = std::sqrt(nr[(size_t)p * 4 + 2]), x2 = std::sqrt(nr[(size_t)p * 4 + 3]);
          lsq_info& I = inf[p];
          I.gmres_its[i] = gs[p].j;
          I.gmres_its_total += gs[p].j;
          I.arnoldi_second_passes += gs[p].nreorth;
          I.gmres_relres[i] = gs[p].relres;
          I.ir_its = i + 1;
          const double dxr = x2 > 0 ? dx / x2 : 0.0, drr = r2 > 0 ? dr / r2 : 0.0;
          I.ir_dx_rel = dxr;
          I.ir_dr_rel = drr;
          I.ir_dx_hist[i] = dxr;
          I.ir_dr_hist[i] = drr;
          if (!std::isfinite(x2) || !std::isfinite(r2)) {
            failed[p] = 2;
            active[p] = 0;
            continue;
          }
          if (dx <= u * x2 && dr <= u * r2) {
            conv[p] = 1;
          } else if (b.o.ir_stop == 0 && i >= 1) {
            const double rx = prev_dx[p] > 0 ? dx / prev_dx[p] : 1.0;
            const double rr = prev_dr[p] > 0 ? dr / prev_dr[p] : 1.0;
            if (rx < 0.5 && rr < 0.5 && rx * dx <= 4.0 * u * x2 && rr * dr <= 4.0 * u * r2) conv[p] = 1;
          }
          prev_dx[p] = dx;
          prev_dr[p] = dr;
        }
      }
    };
    std::vector<int> active(np), conv(np, 0);
    for (int p = 0; p < np; ++p) active[p] = failed[p] ? 0 : 1;
    refine(false, active, conv);
    // Sec. 5: re-run from (x_0, r_0) with the FGMRES products in FP64 where kappa < 1/u_s
    std::vector<int> esc(np, 0);
    bool any_esc = false;
    for (int p = 0; p < np; ++p) {
      const double k = b.o.kappa_hint > 0 ? b.o.kappa_hint : kap[p];
      if (active[p] && !conv[p] && !b.o.no_escalate && k < 1.0 / unit_roundoff(u_s)) {
        esc[p] = 1;
        any_esc = true;
      }
    }
    if (any_esc) {
      restart(esc);
      std::vector<int> conv2(np, 0);
      refine(true, esc, conv2);
      for (int p = 0; p < np; ++p) {
        if (!esc[p]) continue;
        conv[p] = conv2[p];
        inf[p].escalated = 1;
        inf[p].flags |= LSQ_INFO_ESCALATED;
      }
    }
    lsq_status worst = LSQ_OK;
    for (int p = 0; p < np; ++p) {
      lsq_status s;
      if (failed[p] == 1) s = LSQ_E_RANK;
      else if (failed[p] == 2) s = LSQ_E_NONFINITE;
      else s = conv[p] ? LSQ_OK : LSQ_NOT_CONVERGED;
      inf[p].ir_converged = conv[p];
      inf[p].status = s;
      if (statuses) statuses[p] = s;
      if (s < 0) worst = s;
      else if (s == LSQ_NOT_CONVERGED && worst == LSQ_OK) worst = LSQ_NOT_CONVERGED;
    }
    (void)worst;
    return LSQ_OK;
  });
}
