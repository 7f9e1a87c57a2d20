// C ABI (include/lsq.h) and host orchestration of Algorithms 1 and 2.
//
// Everything runs on the handle's stream.  Iterative stages keep their
// scalars on the device; the host enqueues iterations in batches and reads a
// small state block once per batch (kernels of an iteration that starts after
// convergence exit immediately).
#include "host.h"

namespace {

// -------------------------------------------------------------- stages
// Pass 1 (column maxima and, for u_w = F32, the FP32 working copy of A).
float* stage_cast(Ctx& c) {
  StageTimer t(c.h, ST_CAST);
  auto* cmax = static_cast<unsigned long long*>(ws(c.h, "cmax", (c.n + 1) * 8, true));
  float* a32 = nullptr;
  if (c.uw == LSQ_F32) a32 = static_cast<float*>(ws(c.h, "a32", (size_t)c.m * c.lda32 * 4));
  L(launch_colmax_a32(c.A, c.lda, c.b, c.m, c.n, cmax, a32, c.lda32, c.h->d_err, c.st));
  return a32;
}

// Alg. 1 (sketch) -> Y (s x (n+1), column-major, FP64).  a32: the FP32 copy of A left by
// stage_cast (or null); the BF16X3 cast reads it.
void stage_sketch(Ctx& c, double* Y, const float* a32) {
  const int fmt = fmt_of(c.us);
  const int64_t ncols = c.n + 1;
  auto* cmax = static_cast<unsigned long long*>(ws(c.h, "cmax", ncols * 8));
  if (c.o.sketch_kind == 1) {   // Sec. 2's sparse sign embedding (exact fixed-point sums)
    StageTimer tt(c.h, ST_SKETCH);
    const int zeta = c.o.sparse_zeta > 0 ? c.o.sparse_zeta : 8;
    const SparsePlan sp = plan_sparse(c.m, ncols, (int)c.s, c.h->num_sms);
    void* work = ws(c.h, "sparse", sparse_workspace(c.m, ncols, (int)c.s, sp.splits));
    KernTimer kt(c.h, K_SKETCH, c.o.timing);
    L(launch_sparse_sketch(sp, c.A, c.lda, c.b, c.m, c.n, (int)c.s, zeta, c.seed, cmax, work, Y, c.st));
    c.h->launches += 5;
    return;
  }
  int* kexp = static_cast<int*>(ws(c.h, "kexp", ncols * 4));
  if (fmt == FMT_F16 || fmt == FMT_BF16 || fmt == FMT_E4M3 || fmt == FMT_BF16X3) {
    SketchPlan p;
    if (!plan_sketch_tc(fmt, c.s, c.m, ncols, c.h->num_sms, &p, c.o.sketch_kchunk))
      throw StatusFail{LSQ_E_UNSUPPORTED};
    if (p.splits > 65535) throw StatusFail{LSQ_E_INVAL};
    const int t = c.o.no_colscale ? -1 : (fmt == FMT_E4M3 ? 7 : 14);
    const int64_t rows = (int64_t)p.ngroups * p.bn;
    void* Bt;
    {
      StageTimer tt(c.h, ST_CAST);
      L(launch_scale_exps(cmax, ncols, t, kexp, c.st));
      Bt = ws(c.h, "bt", bt_bytes(fmt, c.m, rows));
      L(launch_cast_transpose(fmt, c.A, c.lda, c.b, a32, c.lda32, c.m, c.n, kexp, Bt, rows, c.st));
    }
    StageTimer tt(c.h, ST_SKETCH);
    CUtensorMap tm;
    if (!encode_bt_tmap(&tm, Bt, fmt, (int64_t)p.nt * rows, c.m, p.bn / p.nsub, p.rowb))
      throw StatusFail{LSQ_E_UNSUPPORTED};
    float* partial = static_cast<float*>(ws(c.h, "partial", (size_t)p.splits * ncols * p.s_pad * 4));
    const uint32_t cap = sketch_rec_cap(p);
    const int64_t lists = sketch_rec_lists(p);
    // the correction lists grow with s * m * (column groups); past kRecMaxBytes the
    // in-pipeline exact mode (no lists) is used instead
    bool exact = c.o.sketch_exact != 0 || (size_t)lists * cap * 8 > kRecMaxBytes;
    if (!exact) {
      // deferred correction of the near-midpoint entries (timed together with the GEMM)
      auto* rec = static_cast<uint64_t*>(ws(c.h, "sk_rec", (size_t)lists * cap * 8));
      auto* cnt = static_cast<uint32_t*>(ws(c.h, "sk_cnt", (size_t)lists * 4));
      int* ovf = static_cast<int*>(ws(c.h, "sk_ovf", 64));
      CK(cudaMemsetAsync(ovf, 0, 4, c.st));
      {
        KernTimer kt(c.h, K_SKETCH, c.o.timing);
        L(launch_sketch_tc(p, tm, c.seed, partial, c.h->d_err, c.st, rec, cnt, cap));
      }
      {
        KernTimer kt(c.h, K_SKETCH_FIX, c.o.timing);
        L(launch_sketch_fix(p, c.seed, rec, cnt, cap, c.A, c.lda, c.b, kexp, partial, ovf, c.st));
      }
      c.h->launches += 1;
      exact = read_state<int>(c, ovf) != 0;   // a list overflowed: redo in exact mode
    }
    if (exact) {
      KernTimer kt(c.h, K_SKETCH, c.o.timing);
      L(launch_sketch_tc(p, tm, c.seed, partial, c.h->d_err, c.st));
    }
    L(launch_sketch_reduce(partial, false, p.splits, ncols, c.s, p.s_pad, kexp, Y, c.st));
  } else {
    StageTimer tt(c.h, ST_SKETCH);
    const int64_t base = ((c.s + 15) / 16) * ((ncols + 255) / 256);
    int64_t splits = (8 * (int64_t)c.h->num_sms + base - 1) / base;
    const int64_t ksteps = (c.m + 15) / 16;
    if (splits > ksteps) splits = ksteps;
    if (splits < 1) splits = 1;
    const int64_t kchunk = ((ksteps + splits - 1) / splits) * 16;
    splits = (c.m + kchunk - 1) / kchunk;
    const size_t esz = (fmt == FMT_F64) ? 8 : 4;
    void* partial = ws(c.h, "partial", (size_t)splits * ncols * c.s * esz);
    {
      KernTimer kt(c.h, K_SKETCH, c.o.timing);
      L(launch_sketch_cc(fmt, c.A, c.lda, c.b, c.m, c.n, c.s, c.seed, (int)splits, kchunk, partial,
                         c.s, c.st));
    }
    L(launch_sketch_reduce(partial, fmt == FMT_F64, (int)splits, ncols, c.s, c.s, nullptr, Y, c.st));
  }
}

struct RCopies {
  Tri<float> f32;
  Tri<double> f64;
  double* kappa;
  template <typename T>
  const Tri<T>& get() const {
    if constexpr (sizeof(T) == 4) return f32;
    else return f64;
  }
};

RCopies stage_prepare_r(Ctx& c, const double* R) {
  RCopies r;
  const int64_t ld32 = tri_ld(c.n, 4), ld64 = tri_ld(c.n, 8);
  const size_t n32 = (size_t)ld32 * c.n, n64 = (size_t)ld64 * c.n;
  const size_t nd = (size_t)((c.n + 31) / 32) * 1024;
  r.f32 = {static_cast<float*>(ws(c.h, "R32", n32 * 4)), static_cast<float*>(ws(c.h, "L32", n32 * 4)),
           static_cast<float*>(ws(c.h, "DU32", nd * 4)), static_cast<float*>(ws(c.h, "DL32", nd * 4)), c.n,
           ld32};
  r.f64 = {static_cast<double*>(ws(c.h, "R64", n64 * 8)), static_cast<double*>(ws(c.h, "L64", n64 * 8)),
           static_cast<double*>(ws(c.h, "DU64", nd * 8)), static_cast<double*>(ws(c.h, "DL64", nd * 8)), c.n,
           ld64};
  r.f32.err = c.h->d_err;
  r.f64.err = c.h->d_err;
  r.kappa = static_cast<double*>(ws(c.h, "kappaR", 8));
  L(launch_prepare_r(R, c.n, &r.f32, &r.f64, r.kappa, c.st));
  c.h->launches += 3;
  return r;
}

// Alg. 1 (QR) -> R (n x n) and c; then x_s = R^-1 c in u_QR.
void stage_qr(Ctx& c, const double* Y, double* R, double* xs, RCopies* rc) {
  {
    StageTimer t(c.h, ST_QR);
    const bool f64 = (c.up == LSQ_F64);
    void* work = ws(c.h, "qrwork", (size_t)c.s * (c.n + 1) * (f64 ? 8 : 4));
    // norms, diag(R), then either tau and T (blocked QR) or n + 1 column flags (FP64 QR)
    const size_t tail = std::max<size_t>((32 + 32 * 32) * 8, (size_t)(c.n + 1) * 4);
    double* aux = static_cast<double*>(ws(c.h, "qraux", (2 * c.n + 8) * 8 + tail));
    unsigned* bar = static_cast<unsigned*>(ws(c.h, "qrbar", 64));
    double* cvec = static_cast<double*>(ws(c.h, "qrc", c.n * 8));
    L(launch_qr(f64, Y, c.s, c.n, work, aux, bar, R, cvec, c.h->d_err, c.h->num_sms, c.st));
    c.h->launches += 2;
    *rc = stage_prepare_r(c, R);
    if (xs) {
      if (f64) L((launch_trsv<double, double, double>(true, rc->f64, cvec, 1.0, xs, nullptr, c.st)));
      else L((launch_trsv<float, double, double>(true, rc->f32, cvec, 1.0, xs, nullptr, c.st)));
    }
  }
}

struct LsqrOut {
  LsqrState st;
};

// Alg. 2 (LSQR start): preconditioned LSQR in working precision W from x0 -> x.
template <typename W>
LsqrState stage_lsqr(Ctx& c, const W* Aw, int64_t ldw, const Tri<W>& tri, const double* x0,
                     double* x) {
  StageTimer tmr(c.h, ST_LSQR);
  const int64_t n = c.n, m = c.m;
  const int64_t nvec = round_up(n, 4) + 4;
  W* bw;
  if constexpr (sizeof(W) == 4) {
    bw = static_cast<W*>(ws(c.h, "b32", m * 4));
    L((launch_axpby<double, double, float>(c.b, 1.0, nullptr, 0.0, bw, m, c.st)));
  } else {
    bw = const_cast<double*>(c.b);
  }
  W* u = static_cast<W*>(ws(c.h, "lsqr_u", m * sizeof(W)));
  W* t = static_cast<W*>(ws(c.h, "lsqr_t", nvec * sizeof(W)));
  W* sv = static_cast<W*>(ws(c.h, "lsqr_s", nvec * sizeof(W)));
  W* vt = static_cast<W*>(ws(c.h, "lsqr_vt", nvec * sizeof(W)));
  W* v = static_cast<W*>(ws(c.h, "lsqr_v", nvec * sizeof(W)));
  W* w = static_cast<W*>(ws(c.h, "lsqr_w", nvec * sizeof(W)));
  W* z = static_cast<W*>(ws(c.h, "lsqr_z", nvec * sizeof(W)));
  for (W* vec : {t, sv, vt, v, w, z}) CK(cudaMemsetAsync(vec, 0, nvec * sizeof(W), c.st));
  W* P = static_cast<W*>(ws(c.h, "pblk", (size_t)c.nblk * n * sizeof(W)));
  double* sq = static_cast<double*>(ws(c.h, "sq", c.nblk * 8));
  double* part = static_cast<double*>(ws(c.h, "part", c.nblk2 * 8));
  LsqrState* dst = static_cast<LsqrState*>(ws(c.h, "lsqr_state", sizeof(LsqrState)));
  const int maxit = c.o.lsqr_maxit > 0 ? c.o.lsqr_maxit : (int)(2 * n);
  LsqrState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = c.tol;
  hs.maxit = maxit;
  std::memcpy(c.h->h_pinned + 2048, &hs, sizeof(hs));
  CK(cudaMemcpyAsync(dst, c.h->h_pinned + 2048, sizeof(hs), cudaMemcpyHostToDevice, c.st));
  L(launch_dot(c.b, c.b, m, part, c.nblk2, &dst->normb, true, c.st));
  c.h->launches += 1;
  // u = b - A x0, A^T u  (t = -x0 so that q = A t + 1 * b)
  L((launch_axpby<double, double, W>(x0, -1.0, nullptr, 0.0, t, n, c.st)));
  L(launch_pass_lsqr_any<W>(Aw, ldw, m, n, t, bw, nullptr, 1.0, u, P, sq, c.nblk, nullptr, c.st));
  L(launch_lsqr_colsum<W>(P, c.nblk, n, sq, dst, true, sv, c.st));
  L(launch_lsqr_step<W>(tri, sv, v, w, z, t, dst, true, c.st));
  auto body = [&]() {
    for (int k = 0; k < kBatch; ++k) {
      const int* dn = &dst->done;
      {
        KernTimer kt(c.h, K_LSQR_PASS, c.o.timing);
        L(launch_pass_lsqr_any<W>(Aw, ldw, m, n, t, u, &dst->cu, 1.0, u, P, sq, c.nblk, dn, c.st));
      }
      L(launch_lsqr_colsum<W>(P, c.nblk, n, sq, dst, false, sv, c.st));
      L(launch_lsqr_step<W>(tri, sv, v, w, z, t, dst, false, c.st));
    }
  };
  // CUDA events cannot be timed inside graphs: with opts.timing the batch is launched directly
  CachedGraph* G = (c.o.timing || c.o.no_graph)
                      ? nullptr
                      : get_graph(c,
                                          graph_key(sizeof(W) == 4 ? "lsqr32" : "lsqr64",
                                                    {PV(Aw), ldw, m, n, PV(t), PV(u), PV(P), PV(sq),
                                                     PV(sv), PV(v), PV(w), PV(z), PV(dst), PV(tri.R),
                                                     PV(tri.L), PV(tri.DU), PV(tri.DL), c.nblk}),
                                          body);
  int done = 0, its = 0;
  LsqrState out{};
  while (!done) {
    const size_t mark0 = c.h->marks.size();
    if (G) launch_graph(c, G);
    else body();
    out = read_state<LsqrState>(c, dst);
    const int ran = std::min(kBatch, out.its - its);
    if (c.o.timing) c.h->marks.resize(mark0 + ran);   // keep the passes that did work
    done = out.done;
    its = out.its;
    if (its > maxit + kBatch) break;  // defensive: the device flag ends the loop
  }
  // x = x0 + R^-1 z
  L((launch_trsv<W, W, W>(true, tri, z, 1.0, t, nullptr, c.st)));
  L((launch_axpby<W, double, double>(t, 1.0, x0, 1.0, x, n, c.st)));
  return out;
}

struct GmOut {
  int its;
  int reorth;
  double relres;
  double dr2, r2, dx2, x2;
};

// Alg. 2 (FGMRES): FGMRES on M_L^-1 Atilde M_R^-1 [dr; dz] = [f; h] (operator
// products in TOP), x0 = 0; r += dr, x += dx.
// With dd (TOP = double), the three products are taken in double-double (the Sec. 5
// re-run for u = double): z = R^-1 v_bot, w_top = alpha v_top + A z, w_bot = R^-T A^T v_top,
// each rounded once to FP64, and the Arnoldi step reads w_top as formed.
template <typename TOP>
GmOut stage_fgmres(Ctx& c, const TOP* Aop, int64_t ldop, const Tri<TOP>& tri, const double* f,
                   const double* hv, double tol, int maxit, double* r, double* x, bool dd = false) {
  static_assert(sizeof(TOP) == 4 || sizeof(TOP) == 8, "FP32 or FP64 products");
  if (dd && sizeof(TOP) != 8) throw StatusFail{LSQ_E_INVAL};
  StageTimer tmr(c.h, ST_FGMRES);
  const int64_t m = c.m, n = c.n, ld = m + n;
  const int ldh = maxit + 1;
  double* V = static_cast<double*>(ws(c.h, "gmV", (size_t)ld * (maxit + 1) * 8));
  TOP* Zb = static_cast<TOP*>(ws(c.h, "gmZ", (size_t)(round_up(n, 4) + 4) * (maxit + 1) * sizeof(TOP)));
  const int64_t ldz = round_up(n, 4) + 4;
  double* wv = static_cast<double*>(ws(c.h, "gmW", ld * 8));
  TOP* az = static_cast<TOP*>(ws(c.h, "gmAz", (m + 8) * sizeof(TOP)));
  float* v32 = (sizeof(TOP) == 4) ? static_cast<float*>(ws(c.h, "gmV32", (m + 8) * 4)) : nullptr;
  // coefficient vector of the pass: the FP32 copy of the current column, or the column itself
  const TOP* vcoef = (sizeof(TOP) == 4) ? reinterpret_cast<const TOP*>(v32) : reinterpret_cast<const TOP*>(V);
  const int64_t vstr = (sizeof(TOP) == 4) ? 0 : ld;
  TOP* P = static_cast<TOP*>(ws(c.h, "gmP", (size_t)c.nblk * n * sizeof(TOP)));
  TOP* sb = static_cast<TOP*>(ws(c.h, "gmS", (round_up(n, 4) + 4) * sizeof(TOP)));
  CK(cudaMemsetAsync(Zb, 0, (size_t)(round_up(n, 4) + 4) * (maxit + 1) * sizeof(TOP), c.st));
  double* zlo = dd ? static_cast<double*>(ws(c.h, "gmZlo", (n + 4) * 8)) : nullptr;
  double* Phi = dd ? static_cast<double*>(ws(c.h, "gmPhi", (size_t)c.nblk * n * 8)) : nullptr;
  double* Plo = dd ? static_cast<double*>(ws(c.h, "gmPlo", (size_t)c.nblk * n * 8)) : nullptr;
  double* th = dd ? static_cast<double*>(ws(c.h, "gmTh", (n + 4) * 8)) : nullptr;
  double* tl = dd ? static_cast<double*>(ws(c.h, "gmTl", (n + 4) * 8)) : nullptr;
  CK(cudaMemsetAsync(sb, 0, (round_up(n, 4) + 4) * sizeof(TOP), c.st));
  double* H = static_cast<double*>(ws(c.h, "gmH", (size_t)ldh * maxit * 8, true));
  double* cs = static_cast<double*>(ws(c.h, "gmcs", (maxit + 1) * 8));
  double* sn = static_cast<double*>(ws(c.h, "gmsn", (maxit + 1) * 8));
  double* g = static_cast<double*>(ws(c.h, "gmg", (maxit + 2) * 8, true));
  double* y = static_cast<double*>(ws(c.h, "gmy", (maxit + 1) * 8));
  double* hh = static_cast<double*>(ws(c.h, "gmhh", (maxit + 2) * 8));
  double* Dp = static_cast<double*>(ws(c.h, "gmDp", (size_t)c.nblk2 * (maxit + 2) * 8));
  double* sqp = static_cast<double*>(ws(c.h, "gmsq", c.nblk2 * 8));
  double* p4 = static_cast<double*>(ws(c.h, "gmp4", 4 * c.nblk2 * 8));
  double* nrm = static_cast<double*>(ws(c.h, "gmnrm", 4 * 8));
  GmState* gst = static_cast<GmState*>(ws(c.h, "gm_state", sizeof(GmState)));
  unsigned* gbar = static_cast<unsigned*>(ws(c.h, "gm_bar", 64));
  CK(cudaMemsetAsync(gbar, 0, 64, c.st));
  auto* gseq = static_cast<unsigned long long*>(ws(c.h, "gm_seq", 64));
  CK(cudaMemsetAsync(gseq, 0, 64, c.st));
  if (c.o.expire_sync) {
    // the arrival count starts where no arrival completes the Arnoldi step's grid sync:
    // its bounded waits run out (a test of the timeout path)
    const unsigned preset = 1u << 30;
    std::memcpy(c.h->h_pinned + 3072, &preset, sizeof(preset));
    CK(cudaMemcpyAsync(gbar, c.h->h_pinned + 3072, sizeof(preset), cudaMemcpyHostToDevice, c.st));
  }
  const uint64_t wait_ns = c.o.wait_limit_us > 0 ? (uint64_t)c.o.wait_limit_us * 1000ull : 0ull;
  GmState hs{};
  hs.tol = tol;
  hs.maxit = maxit;
  std::memcpy(c.h->h_pinned + 2048, &hs, sizeof(hs));
  CK(cudaMemcpyAsync(gst, c.h->h_pinned + 2048, sizeof(hs), cudaMemcpyHostToDevice, c.st));
  L(launch_gm_rhs(f, hv, m, n, V, sqp, c.nblk2, c.st, c.alpha));
  L(launch_gm_init(sqp, c.nblk2, gst, g, c.st));
  L(launch_gm_scale0(V, ld, gst, v32, m, c.nblk2, c.st));
  const int maxc = maxit + 1;
  const int mgs = c.o.arnoldi == 3 ? 2 : (c.o.arnoldi == 2 || (c.o.arnoldi == 0 && ld >= kMgsMinRows)) ? 1 : 0;
  const Tri<double>* tri64 = reinterpret_cast<const Tri<double>*>(&tri);
  auto body = [&]() {
    for (int k = 0; k < kBatch; ++k) {
      const int* dn = &gst->done;
      const int* jp = &gst->j;
      if (dd) {
        {
          KernTimer kt(c.h, K_TRSV, c.o.timing);
          L(launch_dd_trsv(true, *tri64, V + m, nullptr, ld, reinterpret_cast<double*>(Zb), ldz, zlo, dn, jp,
                           c.st));
        }
        {
          KernTimer kt(c.h, K_FGM_PASS, c.o.timing);
          const double* A64 = reinterpret_cast<const double*>(Aop);
          L(launch_dd_rows(A64, ldop, m, n, reinterpret_cast<const double*>(Zb), zlo, ldz, V, c.alpha, ld, nullptr,
                           0.0, 1.0, wv, dn, jp, c.h->num_sms, c.st));
          L(launch_dd_cols(A64, ldop, m, n, V, ld, Phi, Plo, c.nblk, dn, jp, c.st));
        }
        L(launch_dd_colsum(Phi, Plo, c.nblk, n, 1.0, th, tl, dn, c.st));
        {
          KernTimer kt(c.h, K_TRSV, c.o.timing);
          L(launch_dd_trsv(false, *tri64, th, tl, 0, wv + m, 0, nullptr, dn, nullptr, c.st));
        }
        {
          KernTimer kt(c.h, K_ARNOLDI, c.o.timing);
          L(launch_gm_step<double>(V, ld, wv, ld, m, nullptr, gst, maxc, Dp, sqp, hh, H, ldh, cs, sn, g, nullptr,
                                   gbar, c.h->d_err, c.h->num_sms, c.st, wait_ns, c.alpha, mgs, gseq,
                                   c.o.expire_sync));
        }
        continue;
      }
      {
        KernTimer kt(c.h, K_TRSV, c.o.timing);
        L((launch_trsv<TOP, double, TOP>(true, tri, V + m, 1.0, Zb, dn, c.st, jp, ld, ldz)));
      }
      {
        KernTimer kt(c.h, K_FGM_PASS, c.o.timing);
        L(launch_pass_fgm<TOP>(Aop, ldop, m, n, Zb, vcoef, az, P, c.nblk, dn, c.st, jp, ldz, vstr,
                               c.h->d_err));
      }
      L((launch_colsum<TOP, TOP>(P, c.nblk, n, nullptr, 1.0, sb, dn, c.st)));
      {
        KernTimer kt(c.h, K_TRSV, c.o.timing);
        L((launch_trsv<TOP, TOP, double>(false, tri, sb, 1.0, wv + m, dn, c.st)));
      }
      // modified Gram-Schmidt, or classical with a second pass only where the first one
      // lost more than half of ||w||^2 ("twice is enough"); Givens step; new column
      {
        KernTimer kt(c.h, K_ARNOLDI, c.o.timing);
        L(launch_gm_step<TOP>(V, ld, wv, ld, m, az, gst, maxc, Dp, sqp, hh, H, ldh, cs, sn, g, v32, gbar,
                              c.h->d_err, c.h->num_sms, c.st, wait_ns, c.alpha, mgs, gseq, c.o.expire_sync));
      }
    }
  };
  int64_t alpha_bits;
  std::memcpy(&alpha_bits, &c.alpha, 8);
  CachedGraph* G =
      (c.o.timing || c.o.no_graph)
          ? nullptr
          : get_graph(c,
                             graph_key(sizeof(TOP) == 4 ? "fgm32" : (dd ? "fgm64dd" : "fgm64"),
                                       {PV(Aop), ldop, m, n, maxit, (int64_t)wait_ns, alpha_bits, PV(V), PV(Zb),
                                        PV(wv), PV(P), PV(zlo), PV(Phi), PV(Plo), PV(th), PV(tl),
                                        PV(az), PV(v32),
                                        PV(sb), PV(H), PV(cs), PV(sn), PV(g), PV(hh), PV(Dp), PV(sqp),
                                        PV(gst), PV(gbar), PV(tri.R), PV(tri.L), PV(tri.DU), PV(tri.DL), c.nblk,
                                        c.nblk2, (int64_t)mgs, PV(gseq), (int64_t)c.o.expire_sync}),
                             body);
  int j = 0;
  GmState out{};
  while (true) {
    const size_t mark0 = c.h->marks.size();
    if (G) launch_graph(c, G);
    else body();
    out = read_state<GmState>(c, gst);
    const int ran = std::min(kBatch, out.j - j);
    if (c.o.timing) {   // keep the marks of the iterations that did work (same count per iteration)
      const size_t per_it = (c.h->marks.size() - mark0) / kBatch;
      c.h->marks.resize(mark0 + (size_t)ran * per_it);
    }
    j = out.j;
    if (out.done || j >= maxit) break;
  }
  check_dev_error(c.h);   // an expired wait ends the solve here (its iterate is not used)
  StageTimer tu(c.h, ST_UPDATE);
  L(launch_gm_solve(gst, H, ldh, g, y, c.st));
  L(launch_gm_apply<double>(V, ld, m, gst, y, r, p4, p4 + c.nblk2, c.nblk2, c.st, c.alpha));   // dr = alpha V_top y
  L(launch_gm_apply<TOP>(Zb, ldz, n, gst, y, x, p4 + 2 * c.nblk2, p4 + 3 * c.nblk2, c.nblk2, c.st));
  for (int k = 0; k < 4; ++k) L(launch_sum_partials(p4 + k * c.nblk2, c.nblk2, nrm + k, true, c.st));
  double hn[4];
  CK(cudaMemcpyAsync(c.h->h_pinned, nrm, 32, cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  std::memcpy(hn, c.h->h_pinned, 32);
  GmOut go;
  go.its = out.j;
  go.reorth = out.nreorth;
  go.relres = out.relres;
  go.dr2 = hn[0];
  go.r2 = hn[1];
  go.dx2 = hn[2];
  go.x2 = hn[3];
  return go;
}

// The refinement loop of Alg. 2 from (x0, r0), FGMRES products in TOP.
// Alg. 2 (refinement residual): f = b - r - A x and g = -A^T r in u_r (FP64, or double-double
// rounded once to FP64; with glo, g is left as the double-double gv + glo).
void stage_residual(Ctx& c, const double* x, const double* r, double* f, double* gv, double* glo = nullptr) {
  const int64_t m = c.m, n = c.n;
  double* P = static_cast<double*>(ws(c.h, "respblk", (size_t)c.nblk * n * 8));
  if (c.ur == LSQ_F64X2) {
    double* Plo = static_cast<double*>(ws(c.h, "respblk_lo", (size_t)c.nblk * n * 8));
    KernTimer kt(c.h, K_RES_PASS, c.o.timing);
    L(launch_dd_rows(c.A, c.lda, m, n, x, nullptr, 0, c.b, 1.0, 0, r, -1.0, -1.0, f, nullptr, nullptr,
                     c.h->num_sms, c.st));
    L(launch_dd_cols(c.A, c.lda, m, n, r, 0, P, Plo, c.nblk, nullptr, nullptr, c.st));
    L(launch_dd_colsum(P, Plo, c.nblk, n, -1.0, gv, glo, nullptr, c.st));
  } else {
    {
      KernTimer kt(c.h, K_RES_PASS, c.o.timing);
      L(launch_pass_res(c.A, c.lda, m, n, x, r, c.b, f, P, c.nblk, c.st));
    }
    L((launch_colsum<double, double>(P, c.nblk, n, nullptr, 1.0, gv, nullptr, c.st)));
  }
}

// dd: FGMRES products in double-double (TOP = double); gmax_min raises the FGMRES cap.
template <typename TOP>
bool stage_refine(Ctx& c, const TOP* Aop, int64_t ldop, const RCopies& rc, double* x, double* r,
                  lsq_info* info, bool dd = false, int gmax_min = 0) {
  const int64_t m = c.m, n = c.n;
  double* f = static_cast<double*>(ws(c.h, "ir_f", m * 8));
  double* gv = static_cast<double*>(ws(c.h, "ir_g", (n + 4) * 8));
  double* hv = static_cast<double*>(ws(c.h, "ir_h", (n + 4) * 8));
  const int irmax = c.o.ir_maxit > 0 ? c.o.ir_maxit : 30;
  const int gmax = std::max(c.o.gmres_maxit > 0 ? c.o.gmres_maxit : 50, gmax_min);
  const double gtol = c.o.gmres_tol > 0 ? c.o.gmres_tol : c.tol;
  const double u = unit_roundoff(c.uw);
  info->aug_alpha = c.alpha;
  bool converged = false;
  double prev_dx = 0.0, prev_dr = 0.0;
  info->ir_its = 0;
  info->gmres_its_total = 0;
  for (int i = 0; i < irmax; ++i) {
    {
      StageTimer t(c.h, ST_RES);
      if (c.ur == LSQ_F64X2 && c.o.h_in_ur) {   // h = R^-T g in u_r (double-double), rounded
        double* glo = static_cast<double*>(ws(c.h, "ir_glo", (n + 4) * 8));
        stage_residual(c, x, r, f, gv, glo);
        L(launch_dd_trsv(false, rc.f64, gv, glo, 0, hv, 0, nullptr, nullptr, nullptr, c.st));
      } else {
        stage_residual(c, x, r, f, gv);
        L((launch_trsv<double, double, double>(false, rc.f64, gv, 1.0, hv, nullptr, c.st)));
      }
    }
    GmOut go = stage_fgmres<TOP>(c, Aop, ldop, rc.get<TOP>(), f, hv, gtol, gmax, r, x, dd);
    info->gmres_its[i] = go.its;
    info->gmres_its_total += go.its;
    info->arnoldi_second_passes += go.reorth;
    info->ir_its = i + 1;
    const double dxr = go.x2 > 0 ? go.dx2 / go.x2 : 0.0;
    const double drr = go.r2 > 0 ? go.dr2 / go.r2 : 0.0;
    info->ir_dx_rel = dxr;
    info->ir_dr_rel = drr;
    info->ir_dx_hist[i] = dxr;
    info->ir_dr_hist[i] = drr;
    info->gmres_relres[i] = go.relres;
    if (!std::isfinite(go.x2) || !std::isfinite(go.r2)) throw StatusFail{LSQ_E_NONFINITE};
    if (go.dx2 <= u * go.x2 && go.dr2 <= u * go.r2) {
      converged = true;
      break;
    }
    if (c.o.ir_stop == 0 && i >= 1) {
      // contraction estimate: the remaining error is about rho times this
      // correction; accept it at the 4u level Sec. 5 asks of the forward errors
      const double rx = prev_dx > 0 ? go.dx2 / prev_dx : 1.0;
      const double rr = prev_dr > 0 ? go.dr2 / prev_dr : 1.0;
      if (rx < 0.5 && rr < 0.5 && rx * go.dx2 <= 4.0 * u * go.x2 && rr * go.dr2 <= 4.0 * u * go.r2) {
        converged = true;
        break;
      }
    }
    prev_dx = go.dx2;
    prev_dr = go.dr2;
  }
  return converged;
}

// Common front part of lsq_lsqr / lsq_lsir: sketch + QR (or R_in), LSQR.
struct Front {
  RCopies rc;
  double* x0;       // start of LSQR (x_s or x0_in or 0)
  float* a32;
  LsqrState ls;
};

Front run_front(Ctx& c, double* x, lsq_info* info) {
  Front fr{};
  fr.a32 = stage_cast(c);
  double* R;
  fr.x0 = static_cast<double*>(ws(c.h, "x0", (c.n + 4) * 8));
  if (c.o.R_in) {
    R = const_cast<double*>(c.o.R_in);
    fr.rc = stage_prepare_r(c, R);
    if (c.o.x0_in) CK(cudaMemcpyAsync(fr.x0, c.o.x0_in, c.n * 8, cudaMemcpyDeviceToDevice, c.st));
    else CK(cudaMemsetAsync(fr.x0, 0, c.n * 8, c.st));
  } else if (c.us == LSQ_AUTO && !c.o.Y_in) {
    // Sec. 3.4 / Sec. 6: choose u_s with kappa(A) u_s < 1.  kappa(A) is estimated by
    // kappa_est(R) = max|r_ii| / min|r_ii| of the sketch just taken (a lower bound,
    // 3 to 30 times below kappa(R) on geometric spectra); a sketch in u_s of an A with
    // kappa(A) > 1/u_s is regularised and its R saturates at a few times 1/u_s, where
    // kappa_est u_s came out 1 to 3.  The test kappa_est u_s < 1/4 accepts the good
    // regime with that margin and rejects the saturated one.  Ladder: BF16, the
    // three-term BF16 split (single), FP64.
    double* Yw = static_cast<double*>(ws(c.h, "Y", (size_t)c.s * (c.n + 1) * 8));
    R = static_cast<double*>(ws(c.h, "R", (size_t)c.n * c.n * 8));
    for (const lsq_prec f : {LSQ_BF16, LSQ_BF16X3, LSQ_F64}) {
      c.us = f;
      info->sketches += 1;
      stage_sketch(c, Yw, fr.a32);
      stage_qr(c, Yw, R, fr.x0, &fr.rc);
      const double k = read_scalar(c, fr.rc.kappa);
      check_dev_error(c.h);
      if (!(k < INFINITY) || k * unit_roundoff(f) < 0.25) break;
    }
    if (c.o.x0_in) CK(cudaMemcpyAsync(fr.x0, c.o.x0_in, c.n * 8, cudaMemcpyDeviceToDevice, c.st));
  } else {
    const double* Y = c.o.Y_in;
    if (!Y) {
      double* Yw = static_cast<double*>(ws(c.h, "Y", (size_t)c.s * (c.n + 1) * 8));
      stage_sketch(c, Yw, fr.a32);
      Y = Yw;
      info->sketches += 1;
    }
    R = static_cast<double*>(ws(c.h, "R", (size_t)c.n * c.n * 8));
    stage_qr(c, Y, R, fr.x0, &fr.rc);
    if (c.o.x0_in) CK(cudaMemcpyAsync(fr.x0, c.o.x0_in, c.n * 8, cudaMemcpyDeviceToDevice, c.st));
  }
  info->us_used = (int32_t)c.us;
  const double kap = read_scalar(c, fr.rc.kappa);
  check_dev_error(c.h);   // a NaN or an infinity in A or b (column-max pass)
  info->kappa_R_est = kap;
  if (!(kap < INFINITY)) throw StatusFail{LSQ_E_RANK};
  if (c.us != LSQ_AUTO && kap * unit_roundoff(c.us) >= 1.0) info->flags |= LSQ_WARN_COND;
  if (c.uw == LSQ_F32)
    fr.ls = stage_lsqr<float>(c, fr.a32, c.lda32, fr.rc.f32, fr.x0, x);
  else
    fr.ls = stage_lsqr<double>(c, c.A, c.lda, fr.rc.f64, fr.x0, x);
  info->lsqr_its = fr.ls.its;
  info->lsqr_flag = fr.ls.flag;
  info->lsqr_normr = fr.ls.normr;
  info->lsqr_normar = fr.ls.normar;
  info->lsqr_normA = fr.ls.normA;
  return fr;
}

// FP64 products stream A in 16-byte pieces: an odd row stride (or an unaligned A)
// gets an even-stride, zero-padded copy first
const double* a64_rows(Ctx& c, int64_t* ld) {
  if ((reinterpret_cast<uintptr_t>(c.A) & 15) == 0 && c.lda % 2 == 0) {
    *ld = c.lda;
    return c.A;
  }
  const int64_t lp = round_up(c.n, 2);
  double* Ap = static_cast<double*>(ws(c.h, "A64p", (size_t)c.m * lp * 8));
  CK(cudaMemsetAsync(Ap, 0, (size_t)c.m * lp * 8, c.st));
  CK(cudaMemcpy2DAsync(Ap, lp * 8, c.A, c.lda * 8, c.n * 8, c.m, cudaMemcpyDeviceToDevice, c.st));
  *ld = lp;
  return Ap;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

size_t lsq_sizeof(int which) {
  if (which == 0) return sizeof(lsq_opts);
  if (which == 1) return sizeof(lsq_info);
  return 0;
}

void lsq_opts_default(lsq_opts* o) {
  if (o) std::memset(o, 0, sizeof(*o));
}

const char* lsq_status_string(lsq_status st) {
  switch (st) {
    case LSQ_OK: return "LSQ_OK";
    case LSQ_NOT_CONVERGED: return "LSQ_NOT_CONVERGED";
    case LSQ_E_INVAL: return "LSQ_E_INVAL";
    case LSQ_E_RANK: return "LSQ_E_RANK";
    case LSQ_E_BREAKDOWN: return "LSQ_E_BREAKDOWN";
    case LSQ_E_NONFINITE: return "LSQ_E_NONFINITE";
    case LSQ_E_CUDA: return "LSQ_E_CUDA";
    case LSQ_E_TIMEOUT: return "LSQ_E_TIMEOUT";
    case LSQ_E_NOMEM: return "LSQ_E_NOMEM";
    case LSQ_E_UNSUPPORTED: return "LSQ_E_UNSUPPORTED";
    case LSQ_E_SIZE: return "LSQ_E_SIZE";
  }
  return "LSQ_UNKNOWN";
}

const char* lsq_last_cuda_error(const lsq_handle* h) { return h ? h->last_cuda.c_str() : ""; }

lsq_status lsq_create(lsq_handle** out, void* cuda_stream) {
  if (!out) return LSQ_E_INVAL;
  *out = nullptr;
  auto* h = new (std::nothrow) lsq_handle();
  if (!h) return LSQ_E_NOMEM;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LSQ_E_CUDA;
  }
  h->user_stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LSQ_E_CUDA;
  }
  if (cudaMalloc(&h->d_err, 64) != cudaSuccess || cudaMemset(h->d_err, 0, 64) != cudaSuccess ||
      cudaMallocHost(&h->h_pinned, 4096) != cudaSuccess) {
    cudaGetLastError();
    if (h->d_err) cudaFree(h->d_err);
    cudaStreamDestroy(h->stream);
    delete h;
    return LSQ_E_NOMEM;
  }
  *out = h;
  return LSQ_OK;
}

lsq_status lsq_destroy(lsq_handle* h) {
  if (!h) return LSQ_E_INVAL;
  cudaStreamSynchronize(h->stream);
  for (auto* w : h->workers) lsq_destroy(w);
  h->workers.clear();
  for (auto& kv : h->graphs) delete kv.second;
  h->graphs.clear();
  for (auto& kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (auto e : h->events) cudaEventDestroy(e);
  if (h->d_err) cudaFree(h->d_err);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return LSQ_OK;
}

lsq_status lsq_sketch(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                      lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                      const lsq_opts* opts, double* Y) {
  Ctx c = make_ctx(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts);
  lsq_status v = validate(c, true);
  if (v != LSQ_OK) return v;
  if (!Y || u_s == LSQ_AUTO) return LSQ_E_INVAL;   // AUTO needs the QR that follows the sketch
  // the FP32 working copy is formed only where the BF16X3 cast reads it
  if (!(u_s == LSQ_BF16X3 && u_w == LSQ_F32)) c.uw = LSQ_F64;
  return run_guarded(h, nullptr, [&]() {
    const float* a32 = stage_cast(c);
    stage_sketch(c, Y, a32);
    return LSQ_OK;
  });
}

lsq_status lsq_qr_r(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                    lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                    const lsq_opts* opts, double* R, double* xs) {
  Ctx c = make_ctx(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts);
  if (c.o.Y_in && !c.A) c.A = c.o.Y_in;  // A is not read when Y is given
  lsq_status v = validate(c, !c.o.Y_in);
  if (v != LSQ_OK) return v;
  if (u_s == LSQ_AUTO && !c.o.Y_in) return LSQ_E_INVAL;   // the precision choice needs lsq_lsqr/lsq_lsir
  return run_guarded(h, nullptr, [&]() {
    const double* Y = c.o.Y_in;
    if (!Y) {
      c.uw = LSQ_F64;
      stage_cast(c);
      double* Yw = static_cast<double*>(ws(c.h, "Y", (size_t)c.s * (c.n + 1) * 8));
      stage_sketch(c, Yw, nullptr);
      Y = Yw;
    }
    double* Rw = R ? R : static_cast<double*>(ws(c.h, "R", (size_t)c.n * c.n * 8));
    RCopies rc;
    stage_qr(c, Y, Rw, xs, &rc);
    const double kap = read_scalar(c, rc.kappa);
    if (!(kap < INFINITY)) return LSQ_E_RANK;
    return LSQ_OK;
  });
}

lsq_status lsq_lsqr(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                    lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                    const lsq_opts* opts, double* x, lsq_info* info) {
  Ctx c = make_ctx(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts);
  lsq_status v = validate(c, true);
  if (v != LSQ_OK) return v;
  if (!x) return LSQ_E_INVAL;
  lsq_info local;
  lsq_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  return run_guarded(h, inf, [&]() {
    StageTimer tt(c.h, ST_TOTAL);
    Front fr = run_front(c, x, inf);
    return fr.ls.flag != 0 ? LSQ_OK : LSQ_NOT_CONVERGED;
  });
}

lsq_status lsq_lsir(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                    lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                    const lsq_opts* opts, double* x, double* r, lsq_info* info) {
  Ctx c = make_ctx(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts);
  lsq_status v = validate(c, true);
  if (v != LSQ_OK) return v;
  if (!x) return LSQ_E_INVAL;
  lsq_info local;
  lsq_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  return run_guarded(h, inf, [&]() {
    StageTimer tt(c.h, ST_TOTAL);
    double* x0 = static_cast<double*>(ws(c.h, "ir_x0", (c.n + 4) * 8));
    Front fr = run_front(c, x0, inf);
    double* rr = r ? r : static_cast<double*>(ws(c.h, "ir_r", c.m * 8));
    double* r0 = static_cast<double*>(ws(c.h, "ir_r0", c.m * 8));
    // r0 = b - A x0 in the working precision (Alg. 2 (initial residual))
    {
      StageTimer t(c.h, ST_RES);
      const int64_t nvec = round_up(c.n, 4) + 4;
      double* sq = static_cast<double*>(ws(c.h, "sq", c.nblk * 8));
      if (c.uw == LSQ_F32) {
        float* t32 = static_cast<float*>(ws(c.h, "lsqr_t", nvec * 4));
        CK(cudaMemsetAsync(t32, 0, nvec * 4, c.st));
        float* q = static_cast<float*>(ws(c.h, "lsqr_u", c.m * 4));
        float* b32 = static_cast<float*>(ws(c.h, "b32", c.m * 4));
        float* P = static_cast<float*>(ws(c.h, "pblk", (size_t)c.nblk * c.n * 4));
        L((launch_axpby<double, double, float>(x0, -1.0, nullptr, 0.0, t32, c.n, c.st)));
        L(launch_pass_lsqr_any<float>(fr.a32, c.lda32, c.m, c.n, t32, b32, nullptr, 1.0, q, P, sq,
                                      c.nblk, nullptr, c.st));
        L((launch_axpby<float, double, double>(q, 1.0, nullptr, 0.0, r0, c.m, c.st)));
      } else {
        double* t64 = static_cast<double*>(ws(c.h, "lsqr_t", nvec * 8));
        CK(cudaMemsetAsync(t64, 0, nvec * 8, c.st));
        double* P = static_cast<double*>(ws(c.h, "pblk", (size_t)c.nblk * c.n * 8));
        L((launch_axpby<double, double, double>(x0, -1.0, nullptr, 0.0, t64, c.n, c.st)));
        L(launch_pass_lsqr_any<double>(c.A, c.lda, c.m, c.n, t64, c.b, nullptr, 1.0, r0, P, sq, c.nblk,
                                       nullptr, c.st));
      }
    }
    CK(cudaMemcpyAsync(x, x0, c.n * 8, cudaMemcpyDeviceToDevice, c.st));
    CK(cudaMemcpyAsync(rr, r0, c.m * 8, cudaMemcpyDeviceToDevice, c.st));
    // FP64 products stream A in 16-byte pieces: an odd row stride (or an unaligned A)
    // gets an even-stride, zero-padded copy first
    auto a64 = [&](int64_t* ld) -> const double* { return a64_rows(c, ld); };
    bool conv;
    if (c.uw == LSQ_F32 && !c.o.ops_escalated) {
      conv = stage_refine<float>(c, fr.a32, c.lda32, fr.rc, x, rr, inf);
    } else {
      int64_t ldp;
      const double* Ap = a64(&ldp);
      conv = stage_refine<double>(c, Ap, ldp, fr.rc, x, rr, inf, c.o.ops_escalated && c.uw == LSQ_F64);
    }
    const double kap = c.o.kappa_hint > 0 ? c.o.kappa_hint : inf->kappa_R_est;
    if (!conv && !c.o.no_escalate && !c.o.ops_escalated && kap < 1.0 / unit_roundoff(c.us)) {
      // Sec. 5: re-run the refinement from (x0, r0) with u_A = u_L = u_R = u^2: FP64 for u
      // single; double-double (the paper's quad) with at most 80 FGMRES iterations for u double
      CK(cudaMemcpyAsync(x, x0, c.n * 8, cudaMemcpyDeviceToDevice, c.st));
      CK(cudaMemcpyAsync(rr, r0, c.m * 8, cudaMemcpyDeviceToDevice, c.st));
      inf->escalated = 1;
      inf->flags |= LSQ_INFO_ESCALATED;
      int64_t ldp;
      const double* Ap = a64(&ldp);
      if (c.uw == LSQ_F32) conv = stage_refine<double>(c, Ap, ldp, fr.rc, x, rr, inf);
      else conv = stage_refine<double>(c, Ap, ldp, fr.rc, x, rr, inf, true, 80);
    }
    inf->ir_converged = conv ? 1 : 0;
    return conv ? LSQ_OK : LSQ_NOT_CONVERGED;
  });
}

lsq_status lsq_ir_step(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                       lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                       const lsq_opts* opts, const double* R, double* x, double* r, lsq_info* info) {
  Ctx c = make_ctx(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts);
  lsq_status v = validate(c, true);
  if (v != LSQ_OK) return v;
  if (!R || !x || !r) return LSQ_E_INVAL;
  c.o.ir_maxit = 1;
  lsq_info local;
  lsq_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  return run_guarded(h, inf, [&]() {
    StageTimer tt(c.h, ST_TOTAL);
    float* a32 = stage_cast(c);
    RCopies rc = stage_prepare_r(c, R);
    const double kap = read_scalar(c, rc.kappa);
    check_dev_error(c.h);   // a NaN or an infinity in A or b
    inf->kappa_R_est = kap;
    if (!(kap < INFINITY)) throw StatusFail{LSQ_E_RANK};
    if (c.uw == LSQ_F32 && !c.o.ops_escalated) {
      stage_refine<float>(c, a32, c.lda32, rc, x, r, inf);
    } else {
      int64_t ldp;
      const double* Ap = a64_rows(c, &ldp);
      stage_refine<double>(c, Ap, ldp, rc, x, r, inf, c.o.ops_escalated && c.uw == LSQ_F64);
    }
    const double gtol = c.o.gmres_tol > 0 ? c.o.gmres_tol : c.tol;
    return inf->gmres_relres[0] <= gtol ? LSQ_OK : LSQ_NOT_CONVERGED;
  });
}

lsq_status lsq_residual(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, lsq_prec u_r,
                        const lsq_opts* opts, const double* x, const double* r, double* f, double* g) {
  Ctx c = make_ctx(h, A, b, m, n, n, LSQ_F64, LSQ_F64, LSQ_F64, u_r, 1.0, 0, opts);
  lsq_status v = validate(c, true);
  if (v != LSQ_OK) return v;
  if (!x || !r || !f || !g) return LSQ_E_INVAL;
  return run_guarded(h, nullptr, [&]() {
    stage_residual(c, x, r, f, g);
    return LSQ_OK;
  });
}

lsq_status lsq_lsir_batched(lsq_handle* h, int32_t nprob, const lsq_problem* probs, lsq_prec u_s,
                            lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol,
                            const lsq_opts* opts, int32_t* statuses, lsq_info* infos) {
  if (opts && (opts->batch_mode < 0 || opts->batch_mode > 1 || opts->batch_grid < 0)) return LSQ_E_INVAL;
  if (!h || nprob < 0 || (nprob > 0 && !probs)) return LSQ_E_INVAL;
  for (int32_t i = 0; i < nprob; ++i) {   // validate everything before any launch
    lsq_opts o;
    if (opts) o = *opts;
    else std::memset(&o, 0, sizeof(o));
    o.lda = probs[i].lda;
    Ctx c = make_ctx(h, probs[i].A, probs[i].b, probs[i].m, probs[i].n, probs[i].s, u_s, u_p, u_w, u_r,
                     tol, probs[i].seed, &o);
    if (validate(c, true) != LSQ_OK || !probs[i].x) return LSQ_E_INVAL;
  }
  if (nprob == 0) return LSQ_OK;
  if (!opts || opts->batch_mode == 0) {
    std::vector<int32_t> stl((size_t)nprob, 0);
    int32_t* stp = statuses ? statuses : stl.data();
    const lsq_status gs = lsq_batch_grouped(h, nprob, probs, u_s, u_p, u_w, u_r, tol, opts, stp, infos);
    if (gs != LSQ_E_UNSUPPORTED) {
      if (gs != LSQ_OK) return gs;
      lsq_status agg = LSQ_OK;
      for (int32_t i = 0; i < nprob; ++i) {
        const lsq_status si = (lsq_status)stp[i];
        if (si < 0 && agg >= 0) agg = si;
        else if (si == LSQ_NOT_CONVERGED && agg == LSQ_OK) agg = LSQ_NOT_CONVERGED;
      }
      return agg;
    }
  }
  const int nw = std::min<int32_t>(nprob, 4);
  while ((int)h->workers.size() < nw) {
    lsq_handle* w = nullptr;
    const lsq_status st = lsq_create(&w, h->user_stream);
    if (st != LSQ_OK) return st;
    h->workers.push_back(w);
  }
  std::atomic<int32_t> next{0};
  std::vector<lsq_status> sts((size_t)nprob, LSQ_OK);
  std::vector<int> who((size_t)nprob, 0);   // worker that ran each problem
  auto work = [&](int k) {
    lsq_handle* w = h->workers[(size_t)k];
    cudaSetDevice(h->device);
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= nprob) break;
      lsq_opts o;
      if (opts) o = *opts;
      else std::memset(&o, 0, sizeof(o));
      o.lda = probs[i].lda;
      if ((double)probs[i].m * (double)probs[i].n < 67108864.0) o.no_graph = 1;
      lsq_info local;
      lsq_info* inf = infos ? &infos[i] : &local;
      who[(size_t)i] = k;
      sts[(size_t)i] = lsq_lsir(w, probs[i].A, probs[i].b, probs[i].m, probs[i].n, probs[i].s, u_s, u_p,
                                u_w, u_r, tol, probs[i].seed, &o, probs[i].x, probs[i].r, inf);
    }
  };
  std::vector<std::thread> threads;
  for (int k = 1; k < nw; ++k) threads.emplace_back(work, k);
  work(0);
  for (auto& t : threads) t.join();
  lsq_status agg = LSQ_OK;
  for (int32_t i = 0; i < nprob; ++i) {
    if (statuses) statuses[i] = sts[(size_t)i];
    if (sts[(size_t)i] < 0 && agg >= 0) {
      agg = sts[(size_t)i];
      if (agg == LSQ_E_CUDA)   // the text of the first failure, on the caller's handle
        h->last_cuda = "problem " + std::to_string(i) + ": " + h->workers[(size_t)who[(size_t)i]]->last_cuda;
    }
    else if (sts[(size_t)i] == LSQ_NOT_CONVERGED && agg == LSQ_OK) agg = LSQ_NOT_CONVERGED;
  }
  return agg;
}

lsq_status lsq_omega(lsq_handle* h, int64_t s, int64_t j0, int64_t cols, lsq_prec u_s, uint64_t seed,
                     double* out) {
  if (!h || !out || s < 1 || cols < 1 || j0 < 0 || s > ((int64_t)1 << 31) || fmt_of(u_s) < 0)
    return LSQ_E_INVAL;
  return run_guarded(h, nullptr, [&]() {
    CK(launch_omega(fmt_of(u_s), s, j0, cols, seed, out, h->stream));
    ++h->launches;
    return LSQ_OK;
  });
}

lsq_status lsq_lsir_host(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
                         lsq_prec u_s, lsq_prec u_p, lsq_prec u_w, lsq_prec u_r, double tol, uint64_t seed,
                         const lsq_opts* opts, double* x, double* r, lsq_info* info) {
  if (!h || !A || !b || !x || n < 1 || m < n || m > ((int64_t)1 << 36)) return LSQ_E_INVAL;
  const int64_t lda = (opts && opts->lda > 0) ? opts->lda : n;
  if (lda < n) return LSQ_E_INVAL;
  const size_t a_elems = (size_t)(m - 1) * (size_t)lda + (size_t)n;   // rows end at column n
  double *dA = nullptr, *db = nullptr, *dx = nullptr, *dr = nullptr;
  try {
    dA = static_cast<double*>(ws(h, "host_A", a_elems * 8));
    db = static_cast<double*>(ws(h, "host_b", (size_t)m * 8));
    dx = static_cast<double*>(ws(h, "host_x", (size_t)n * 8));
    if (r) dr = static_cast<double*>(ws(h, "host_r", (size_t)m * 8));
    // inputs onto the work stream, after whatever the caller's stream has queued
    CK(cudaEventRecord(h->ev_in, h->user_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
    CK(cudaMemcpyAsync(dA, A, a_elems * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(db, b, (size_t)m * 8, cudaMemcpyHostToDevice, h->stream));
  } catch (const CudaFail& f) {
    h->last_cuda = std::string(f.what) + ": " + cudaGetErrorString(f.e);
    cudaGetLastError();
    return LSQ_E_CUDA;
  } catch (const StatusFail& f) {
    return f.st;
  }
  const lsq_status st = lsq_lsir(h, dA, db, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, dx, dr, info);
  if (st != LSQ_OK && st != LSQ_NOT_CONVERGED) return st;
  cudaError_t e = cudaMemcpyAsync(x, dx, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && r) e = cudaMemcpyAsync(r, dr, (size_t)m * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->last_cuda = std::string("lsq_lsir_host result copy: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return LSQ_E_CUDA;
  }
  return st;
}

}  // extern "C"
