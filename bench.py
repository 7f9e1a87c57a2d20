"""Benchmark: time-to-solution of the mixed-precision sketch-and-precondition
least-squares solver on one GB300 (replicas only across GPUs).

Workload (one "step" = one full call of lsq_lsir on data resident in HBM), the
largest configuration that fits one GPU:
  A = U diag(sigma) V^T, m = 4,000,000, n = 1000, kappa = 1e7 (geometric
  sigma from 1 to 1e-7), b = A x + r_perp with ||r_perp|| / ||b|| = 1e-6;
  A in FP64 (32 GB); Gaussian sketch s = 4n on BF16 tensor cores (FP32
  accumulation, power-of-two column scaling), QR in FP64, LSQR in FP32
  (tol 1e-6, <= 2n iterations), FGMRES-LSIR with FP32 products and FP64
  residuals, Arnoldi and Givens (<= 30 refinement steps of <= 50 FGMRES
  iterations).
The sketch precision follows the paper's rule (Sec. 3.4: choose u_s with
kappa(A) u_s < 1): at kappa = 1e7 the single-term BF16 sketch violates it
(kappa u_s = 3.9e4), so the three-term BF16 split (single precision on BF16
tensor cores, u_s = 2^-24, kappa u_s = 0.6) is used; the single-term BF16 run
of the configuration is reported beside it, with capped iterations.
The inputs are drawn on the device (lsq_synth.device); the generator's x and
r_perp stand in for the stored-data solution (they differ from it by about
1e-9 relative here, far below the 4u = 2.4e-7 being checked).

Also reported: per-kernel device times from CUDA events around every launch in
one instrumented solve (events cannot be timed inside CUDA graphs), the
dominant kernel against its roofline, the whole solve against the sum of its
stage floors, the all-FP64 GPU path on the same inputs, the m = 1e5, n = 500,
kappa = 1e6 configuration as a secondary line, an end-to-end number through
lsq_lsir_host with host buffers, SM clocks sampled during the timed region,
and the CPU oracle timed on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solution mixed vs FP64 at fwd err<=u_w bound; sketch TFLOP/s, matvec GB/s"
#: sketch precisions in increasing cost, with their unit roundoff
US_LADDER = [("e4m3", 2.0 ** -4), ("bf16", 2.0 ** -8), ("f16", 2.0 ** -11), ("bf16x3", 2.0 ** -24),
             ("f64", 2.0 ** -53)]


def select_us(kappa):
    """Cheapest sketch precision with kappa(A) u_s < 1 (Sec. 3.4, Sec. 6)."""
    for name, u in US_LADDER:
        if kappa * u < 1.0:
            return name
    return "f64"


WL = dict(workload="randsvd m=4000000 n=1000 kappa=1e7 rho=1e-6; Gaussian sketch s=4n on BF16 tensor "
                   "cores (u_s by kappa*u_s<1), FP64 QR, FP32 LSQR/FGMRES products, FP64 residuals",
          m=4_000_000, n=1000, s=4000, kappa=1e7, rho=1e-6, u_p="f64", u_w="f32", u_r="f64",
          tol=1e-6, seed=0, data_seed=4)
WL["u_s"] = select_us(WL["kappa"])
#: the secondary configuration (m = 1e5, n = 500, kappa = 1e6), also device-drawn
WL2 = dict(m=100_000, n=500, s=2000, kappa=1e6, rho=1e-3, u_p="f32", u_w="f32", u_r="f64", tol=1e-6,
           seed=0, data_seed=1)
WL2["u_s"] = select_us(WL2["kappa"])
CONFIG_EXTRA = dict(l2="inputs larger than L2 (A is 32 GB FP64 plus a 16 GB FP32 copy)",
                    parallelism="replicas", u_s_rule="cheapest u_s with kappa*u_s<1 (Sec. 3.4)",
                    inputs="drawn on the device, resident in HBM when the timed region starts")


def config():
    """The line's config (the same on both arms)."""
    return dict(WL, **CONFIG_EXTRA)
FALLBACK_HBM = 6800.0
#: how the oracle uses the host's cores (numpy: BLAS products on its thread pool)
THREADS_NOTE = ("matrix products on numpy's BLAS thread pool (all cores unless OMP_NUM_THREADS says "
                "otherwise); the Philox/Box-Muller generation and the other elementwise work on one thread")
#: rows of the CPU sample: sketch on M_SKETCH rows, LSQR/FGMRES iterations fitted on two row counts,
#: QR on an s x N_QR block (all scaled to the workload, see oracle_step)
M_SKETCH, M_ITER, N_QR = 1000, (8000, 16000), 250


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return dict(hbm=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]),
                    bf16_sustained=float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), kind="measured")
    except Exception:
        return dict(hbm=FALLBACK_HBM, bf16=1900.0, bf16_sustained=1700.0, kind="fallback")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait for its first sample so the
        # sampled window covers the work that follows
        t0 = time.time()
        while time.time() - t0 < 10 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


#: committed ncu summaries with the DRAM traffic of a kernel (at n = 1000, smaller m)
TRAFFIC_PROFILES = {"fgmres_pass": "pass_bulk_fgmres_m200000_n1000.md"}


def measured_traffic(kernel, m):
    """DRAM bytes per launch (read + write) of `kernel` at m rows, from its committed
    ncu summary (captured on a smaller m and scaled by the rows, the unit the pass
    streams), or None if there is none or the kernel's source changed since."""
    if kernel not in TRAFFIC_PROFILES:
        return None
    path = os.path.join(ROOT, "profiles", TRAFFIC_PROFILES[kernel])
    try:
        text = open(path).read()
        tb = float(re.search(r"^traffic_bytes_per_launch: (\d+)", text, re.M).group(1))
        m_cap = float(re.search(r"^captured_m: (\d+)", text, re.M).group(1))
        srcs = re.findall(r'^source: (\S+)(?: from "(.+?)" to "(.+?)")? sha256\[:16\] ([0-9a-f]+)$', text, re.M)
        if not srcs:
            return None
        for src, start, end, h in srcs:
            body = open(os.path.join(ROOT, src), "rb").read()
            if start:   # the kernel's own region of the file
                t = body.decode()
                i = t.index(start)
                body = t[i:t.index(end, i)].encode()
            if hashlib.sha256(body).hexdigest()[:16] != h:
                return None
    except (OSError, AttributeError, ValueError):
        return None
    return tb * m / m_cap


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(t, world):
    """max over ranks of a float (host), with a barrier."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    v = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- oracle leg
def oracle_sample(seed=4):
    """Host inputs of the CPU sample: rows drawn like the workload (same recipe,
    fewer rows), an R for the iterations, and an s x N_QR block for the QR."""
    from lsq_synth import randsvd_problem
    n, s = WL["n"], WL["s"]
    P = randsvd_problem(max(M_ITER), n, WL["kappa"], rho=WL["rho"], seed=seed)
    g = np.random.default_rng(seed)
    R = np.linalg.qr(g.standard_normal((s, n)) @ np.diag(P.sigma) / np.sqrt(s), mode="r")
    Yq = g.standard_normal((s, min(N_QR, n) + 1)) / np.sqrt(s)
    return dict(A=P.A, b=P.b, R=R, Yq=Yq)


def oracle_step(S, iters):
    """Times the CPU oracle on a bounded sample of the workload; returns (ms_estimate, detail).

    Algorithm 1's sketch (u_s of the workload) on the first M_SKETCH rows, scaled
    linearly to m; the FP64 Householder QR of an s x N_QR block, scaled by the flop
    count n^2 (s - n/3); 4 LSQR and 4 FGMRES iterations (FP32 products) on two row
    counts, fitted as a + b*rows per iteration (the products grow with the rows, the
    triangular solves do not) and taken to m rows and the given iteration counts.
    """
    from oracle import fgmres, lsqr, qr, sketch
    m, n, s = WL["m"], WL["n"], WL["s"]
    A, b, R = S["A"], S["b"], S["R"]
    t0 = time.perf_counter()
    sketch.sketch(A[:M_SKETCH], b[:M_SKETCH], s, WL["seed"], WL["u_s"])
    t1 = time.perf_counter()
    nq = S["Yq"].shape[1] - 1
    qr.householder_qr(S["Yq"], nq, dtype=np.float64)
    t2 = time.perf_counter()
    per = {}
    for rows in M_ITER:
        ta = time.perf_counter()
        lsqr.lsqr(A[:rows], b[:rows], R, np.zeros(n), 0.0, 4, dtype=np.float32)
        tb = time.perf_counter()
        fgmres.fgmres(A[:rows], R, b[:rows], np.zeros(n), 0.0, 4, op_dtype=np.float32)
        tc = time.perf_counter()
        per[rows] = ((tb - ta) / 4, (tc - tb) / 4)
    r0, r1 = M_ITER

    def at_m(k):   # per-iteration seconds at m rows from the two sampled row counts
        slope = max(0.0, (per[r1][k] - per[r0][k]) / (r1 - r0))
        icpt = max(0.0, per[r0][k] - slope * r0)
        return icpt + slope * m

    qr_scale = n * n * (s - n / 3) / (nq * nq * (s - nq / 3))
    est = ((t1 - t0) * m / M_SKETCH + (t2 - t1) * qr_scale + at_m(0) * iters["lsqr"]
           + at_m(1) * iters["fgmres"])
    return est * 1e3, dict(sketch_s=t1 - t0, qr_block_s=t2 - t1, qr_scale=qr_scale,
                           lsqr_per_it_s_at_m=at_m(0), fgmres_per_it_s_at_m=at_m(1),
                           wall_s=time.perf_counter() - t0)


def sample_note(iters):
    return (f"{WL['u_s']} sketch of the first {M_SKETCH} rows (scaled linearly to m={WL['m']}); FP64 "
            f"Householder QR of an s x {N_QR} block (scaled by n^2(s-n/3)); 4 LSQR + 4 FGMRES iterations "
            f"with FP32 products on {M_ITER[0]} and {M_ITER[1]} rows, fitted per iteration as a + b*rows "
            f"and taken to m rows and {iters['lsqr']} LSQR / {iters['fgmres']} FGMRES iterations (the GPU "
            f"solve's counts; a full oracle solve at this size does not fit a bench run)")


#: iteration counts of the GPU's solve of this workload (used when no GPU run is at hand)
GPU_ITERS = {"lsqr": 20, "fgmres": 250}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    S = oracle_sample()
    iters = dict(GPU_ITERS)
    for _ in range(args.warmup):
        oracle_step(S, iters)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, _detail = oracle_step(S, iters)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / args.steps * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3/f32/f64", "data": "synthetic", "config": config(),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "ms", "cores": os.cpu_count(),
                             "threads": THREADS_NOTE, "sample": sample_note(iters)},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched configuration
BATCH = dict(count=512, m_range=(5000, 200000), n_range=(32, 256), kappa_range=(1e2, 1e8),
             rho_range=(1e-8, 1e-1), seed=4)
BATCH_US = "bf16"


def run_batched(lsq, torch, pk, fp64_fma, opts=None, warm=True):
    """The batched configuration: BATCH["count"] problems (m, n, kappa, rho drawn as
    configured) drawn on the device, BF16 sketch s = 4n, FP32 QR/LSQR/FGMRES products,
    FP64 residuals, through one grouped lsq_lsir_batched call on its own handle.  One
    warm-up call (workspace allocation, graph captures), then one timed call (CUDA events
    on the handle's stream, and the host clock).  The roofline fraction sums each problem's
    stage floors times its own iteration counts over the measured time."""
    from lsq_synth.device import DeviceRandsvd
    from lsq_synth.problems import batch_specs
    specs = batch_specs(**BATCH)
    t0 = time.perf_counter()
    probs = []
    for k, sp in enumerate(specs):
        gen = DeviceRandsvd(sp["m"], sp["n"], seed=sp["seed"])
        A, b, _ = gen.problem(sp["kappa"], sp["rho"])
        gen.release()
        del gen
        probs.append(dict(A=A.contiguous(), b=b.contiguous(), m=sp["m"], n=sp["n"], s=4 * sp["n"], seed=k,
                          x=torch.zeros(sp["n"], dtype=torch.float64, device=A.device),
                          r=torch.zeros(sp["m"], dtype=torch.float64, device=A.device)))
    torch.cuda.synchronize()
    t_draw = time.perf_counter() - t0
    hb = lsq.Handle()
    try:
        if warm:
            lsq.lsq_lsir_batched(hb, probs, BATCH_US, "f32", "f32", "f64", 1e-6, opts)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        st, sts, infos = lsq.lsq_lsir_batched(hb, probs, BATCH_US, "f32", "f32", "f64", 1e-6, opts)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        dev_s = e0.elapsed_time(e1) / 1e3
    finally:
        hb.close()
    floor_ms = 0.0
    bytes_passes = 0.0
    its = {"lsqr": 0, "fgmres": 0, "ir": 0, "escalated": 0}
    for sp, inf in zip(specs, infos):
        d = inf.as_dict()
        wl = {"m": sp["m"], "n": sp["n"], "s": 4 * sp["n"], "u_s": BATCH_US, "u_p": "f32"}
        floor_ms += sum(tts_floor(wl, d, pk, fp64_fma).values())
        lda32 = (sp["n"] + 3) // 4 * 4
        bytes_passes += (d["lsqr_its"] + d["gmres_its_total"] + 2) * (4.0 * sp["m"] * lda32 + 8.0 * sp["m"])
        its["lsqr"] += d["lsqr_its"]
        its["fgmres"] += d["gmres_its_total"]
        its["ir"] += d["ir_its"]
        its["escalated"] += d["escalated"]
    t_s = max(wall, dev_s)
    conv = sum(1 for i in infos if i.ir_converged == 1)
    return {"problems": len(specs), "u_s": BATCH_US, "seconds": t_s, "device_seconds": dev_s,
            "solves_per_s": len(specs) / t_s, "converged": conv,
            "not_converged": sum(1 for v in sts if v == 1), "errors": sum(1 for v in sts if v < 0),
            "kappa_u_s_below_1": sum(1 for sp in specs if sp["kappa"] * 2.0 ** -8 < 1.0),
            "iterations_total": its,
            "roofline": {"floor_ms": floor_ms, "frac": floor_ms / (t_s * 1e3),
                         "pass_bytes_gbs": bytes_passes / t_s / 1e9,
                         "how": "sum over the problems of their stage floors (HBM bytes, tensor flops at the "
                                "sustained BF16 peak, FP64 FMAs at the measured FP64 rate) times their own "
                                "iteration counts, over the measured time of the call"},
            "mode": ("per problem (four streams, lsq_lsir on each)" if opts and opts.get("batch_mode")
                     else "grouped (one launch per stage for all problems, iteration batches as CUDA graphs)"),
            "draw_s": t_draw,
            "sample": "m ~ U[5000, 200000], n ~ U[32, 256], kappa log-U[1e2, 1e8], rho log-U[1e-8, 1e-1], "
                      "s = 4n, drawn on the device (U from CholeskyQR2 of a Gaussian); inputs resident; "
                      "timed: one lsq_lsir_batched call after a warm-up call"}


# ---------------------------------------------------------------- rooflines
def kernel_work(wl, d, fp64_fma):
    """Algorithmic work and floor (ms) of each timed kernel of one solve (info dict d)."""
    m, n, s = wl["m"], wl["n"], wl["s"]
    lda32 = (n + 3) // 4 * 4
    terms = 3 if wl["u_s"] == "bf16x3" else 1
    its = d["gmres_its"]
    # Arnoldi: a classical Gram-Schmidt pass (h = V^T w, w -= V h) against j + 1 basis
    # vectors at step j; the steps that ran the second pass counted at the average cost
    # of a step (the library reports their number, not their j)
    arn_fma = sum(2.0 * (j + 1) * (m + n) for k in its for j in range(k))
    tot_its = max(1, sum(its))
    arn_fma *= 1.0 + d.get("arnoldi_second_passes", 0) / tot_its
    return {"sketch_gemm": {"flop": 2.0 * s * m * (n + 1) * terms, "bound": "tensor"},
            "lsqr_pass": {"bytes": 4.0 * m * lda32 + 8.0 * m, "bound": "hbm"},
            "fgmres_pass": {"bytes": 4.0 * m * lda32 + 8.0 * m, "bound": "hbm"},
            "residual_pass": {"bytes": 8.0 * m * n + 32.0 * m, "fma": 2.0 * m * n, "bound": "fp64"},
            "arnoldi_step": {"fma_total": arn_fma, "bound": "fp64"}}


def tts_floor(wl, d, pk, fp64_fma):
    """Sum over the solve's stages of each stage's floor times the iteration counts it ran
    (ms): cast (HBM), sketch (tensor pipe), QR (FP64 pipe), LSQR passes (HBM), residual
    passes (the larger of HBM and the FP64 pipe), FGMRES passes (HBM) and Arnoldi steps
    (FP64 pipe).  Triangular solves and small kernels are left out (latency-bound)."""
    m, n, s = wl["m"], wl["n"], wl["s"]
    hbm = pk["hbm"] * 1e9
    lda32 = (n + 3) // 4 * 4
    terms = 3 if wl["u_s"] == "bf16x3" else 1
    up64 = wl["u_p"] == "f64"
    f = {}
    f["cast"] = (8.0 * m * n + 4.0 * m * lda32 + 2.0 * terms * m * (n + 1)) / hbm
    f["sketch"] = 2.0 * s * m * (n + 1) * terms / (pk["bf16_sustained"] * 1e12)
    qr_fma = n * n * (s - n / 3.0)
    f["qr"] = qr_fma / fp64_fma if up64 else 0.0
    f["lsqr"] = (d["lsqr_its"] + 1) * (4.0 * m * lda32 + 8.0 * m) / hbm
    nres = d["ir_its"] + 1
    f["residual"] = nres * max((8.0 * m * n + 32.0 * m) / hbm, 2.0 * m * n / fp64_fma)
    tot_its = d["gmres_its_total"]
    f["fgmres_pass"] = tot_its * (4.0 * m * lda32 + 8.0 * m) / hbm
    arn = sum(2.0 * (j + 1) * (m + n) for k in d["gmres_its"] for j in range(k))
    arn *= 1.0 + d.get("arnoldi_second_passes", 0) / max(1, tot_its)
    f["arnoldi"] = arn / fp64_fma
    return {k: v * 1e3 for k, v in f.items()}


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2410_06319_gb300 as lsq
    from lsq_synth.device import DeviceRandsvd

    pk = peaks()
    fp64_fma = lsq.lsq_probe_fma_rate("f64")
    m, n, s = WL["m"], WL["n"], WL["s"]
    t_draw = time.time()
    gen = DeviceRandsvd(m, n, seed=WL["data_seed"])
    A, b, rperp = gen.problem(WL["kappa"], WL["rho"])
    x_true = gen.x_true.clone()
    gen.release()
    del gen
    torch.cuda.empty_cache()
    t_draw = time.time() - t_draw
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    h = lsq.Handle()
    stream = torch.cuda.current_stream()
    rest = (WL["u_p"], WL["u_w"], WL["u_r"], WL["tol"], WL["seed"])

    def solve(opts=None, AA=A, bb=b, xx=x, rr=r, us=WL["u_s"], mm=m, nn=n, ss=s, rst=rest):
        return lsq.lsq_lsir(h, AA, bb, mm, nn, ss, us, *rst, opts, xx, rr)

    def fe(xx, rr, xt, rp):
        return ((torch.linalg.norm(xx - xt) / torch.linalg.norm(xt)).item(),
                (torch.linalg.norm(rr - rp) / torch.linalg.norm(rp)).item())

    for _ in range(args.warmup):
        solve()
    # ---- timed region: K full solves (CUDA graphs inside the library)
    clk = Clocks(local)
    infos = []
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        st, info = solve()
        infos.append(info.as_dict())
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    clocks["window"] = "timed solves"
    barrier(world)
    t_ms = ev0.elapsed_time(ev1)
    t_ms = barrier_max(t_ms, world)
    value = t_ms / (args.steps * world)       # ms per solve, whole job
    last = infos[-1]
    fe_mixed = fe(x, r, x_true, rperp)

    # ---- one instrumented solve: CUDA events around every kernel launch of the path
    st_t, info_t = solve({"timing": 1})
    d = info_t.as_dict()
    tot = d["kern_ms"]
    cnt = d["kern_launches"]
    solve_ms = d["stage_ms"]["total"]
    kernels = {k: {"launches": cnt[k], "total_ms": tot[k], "avg_us": tot[k] / cnt[k] * 1e3,
                   "share_of_solve": tot[k] / solve_ms if solve_ms > 0 else None}
               for k in lsq.KERNELS if cnt.get(k)}
    work = kernel_work(WL, d, fp64_fma)
    for k, kw in work.items():
        if k not in kernels:
            continue
        kk = kernels[k]
        avg_s = kk["avg_us"] * 1e-6
        if "bytes" in kw:
            kk["bytes_per_launch"] = kw["bytes"]
            kk["gbs"] = kw["bytes"] / avg_s / 1e9
            kk["frac_hbm"] = kk["gbs"] / pk["hbm"]
        if "flop" in kw:
            kk["flop_per_launch"] = kw["flop"]
            kk["tflops"] = kw["flop"] / avg_s / 1e12
            kk["tflops_method"] = 2.0 * s * m * (n + 1) / avg_s / 1e12
            kk["frac_bf16_sustained"] = kk["tflops"] / pk["bf16_sustained"]
        if "fma" in kw:
            kk["fp64_fma_per_s"] = kw["fma"] / avg_s
            kk["frac_fp64"] = kk["fp64_fma_per_s"] / fp64_fma
        if "fma_total" in kw:
            kk["fp64_fma_per_s"] = kw["fma_total"] / (kk["total_ms"] * 1e-3)
            kk["frac_fp64"] = kk["fp64_fma_per_s"] / fp64_fma
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    kd = kernels[dom]
    if dom in ("fgmres_pass", "lsqr_pass"):
        roofline = {"bound": "hbm", "kernel": dom, "achieved": kd["gbs"], "peak": pk["hbm"],
                    "peak_kind": pk["kind"], "unit": "GB/s", "frac": kd["frac_hbm"],
                    "traffic": measured_traffic(dom, m), "algorithmic_bytes_per_launch": kd["bytes_per_launch"]}
    elif dom == "sketch_gemm":
        roofline = {"bound": "tensor", "kernel": dom, "achieved": kd["tflops"], "peak": pk["bf16_sustained"],
                    "peak_kind": pk["kind"] + " sustained", "unit": "TFLOP/s", "frac": kd["frac_bf16_sustained"],
                    "traffic": None}
    else:
        roofline = {"bound": "alu", "kernel": dom, "achieved": kd.get("fp64_fma_per_s", 0) * 2e-12,
                    "peak": fp64_fma * 2e-12, "peak_kind": "FP64 FMA rate measured by lsq_probe_fma_rate",
                    "unit": "TFLOP/s", "frac": kd.get("frac_fp64"), "traffic": None}
    roofline["how"] = ("CUDA events around each launch in one instrumented solve (same kernels and "
                       "arguments as the timed solves); kernel chosen by its total device time per solve")
    floors = tts_floor(WL, d, pk, fp64_fma)
    tts_roof = {"floor_ms": floors, "floor_total_ms": sum(floors.values()), "measured_ms": value,
                "frac": sum(floors.values()) / value,
                "how": "stage floors (HBM bytes, tensor flops at the sustained BF16 peak, FP64 FMAs at the "
                       "measured FP64 rate) times the iteration counts of the solve, over its measured time"}

    # ---- the configuration's literal single-term BF16 sketch (kappa u_s = 3.9e4: outside Sec. 3)
    single = {}
    for us in ("bf16",):
        xs_, rs_ = torch.zeros_like(x), torch.zeros_like(r)
        o = {"lsqr_maxit": 400, "ir_maxit": 3, "no_escalate": 1}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st1, i1 = solve(o, xx=xs_, rr=rs_, us=us)
        e1.record(stream)
        torch.cuda.synchronize()
        d1 = i1.as_dict()
        fx, fr = fe(xs_, rs_, x_true, rperp)
        single[us] = {"ms": e0.elapsed_time(e1), "caps": o, "converged": bool(d1["ir_converged"]),
                      "lsqr_its": d1["lsqr_its"], "ir_its": d1["ir_its"],
                      "fgmres_total": d1["gmres_its_total"], "kappa_R_est": d1["kappa_R_est"],
                      "fe_x": fx, "fe_r": fr}
        del xs_, rs_

    # ---- the sparse sign embedding (Sec. 2) as the sketch, same workload and solver settings
    sparse_leg = {}
    try:
        xs_, rs_ = torch.zeros_like(x), torch.zeros_like(r)
        o = {"sketch_kind": 1}
        solve(o, xx=xs_, rr=rs_)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ksp = max(1, min(3, args.steps))
        e0.record(stream)
        for _ in range(ksp):
            stp, ip = solve(o, xx=xs_, rr=rs_)
        e1.record(stream)
        torch.cuda.synchronize()
        stq, iq = solve(dict(o, timing=1), xx=xs_, rr=rs_)
        dq = iq.as_dict()
        fx, fr = fe(xs_, rs_, x_true, rperp)
        sparse_leg = {"tts_ms": e0.elapsed_time(e1) / ksp, "sketch_ms": dq["kern_ms"]["sketch_gemm"],
                      "sketch_stage_ms": dq["stage_ms"]["sketch"], "zeta": 8, "converged": bool(dq["ir_converged"]),
                      "iterations": {"lsqr": dq["lsqr_its"], "ir": dq["ir_its"], "fgmres_total": dq["gmres_its_total"]},
                      "fe_x": fx, "fe_r": fr, "meets_bound": bool(max(fx, fr) <= 4 * 2.0 ** -24),
                      "sketch_gbs": 8.0 * m * (n + 1) / (dq["kern_ms"]["sketch_gemm"] * 1e-3) / 1e9
                      if dq["kern_ms"]["sketch_gemm"] > 0 else None,
                      "how": "lsq_lsir with opts.sketch_kind = 1 (zeta = 8 signed rows per data row, exact "
                             "fixed-point sums); everything else as the headline solve"}
        del xs_, rs_
    except Exception as exc:
        sparse_leg = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- all-FP64 GPU path on the same inputs: FP64 sketch, QR and LSQR
    fp64 = {}
    try:
        Yfull = torch.zeros(s * (n + 1), dtype=torch.float64, device="cuda")
        lsq.lsq_sketch(h, A, b, m, n, s, WL["u_s"], *rest, None, Yfull)
        frac = 20
        ms_ = m // frac
        Ys = torch.zeros_like(Yfull)
        As, bs = A[:ms_], b[:ms_]
        lsq.lsq_sketch(h, As, bs, ms_, n, s, "f64", "f64", "f64", "f64", 1e-10, WL["seed"], None, Ys)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lsq.lsq_sketch(h, As, bs, ms_, n, s, "f64", "f64", "f64", "f64", 1e-10, WL["seed"], None, Ys)
        e1.record(stream)
        torch.cuda.synchronize()
        sk64 = e0.elapsed_time(e1) * (m / ms_)
        R64 = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        xs64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        x64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        lsq.lsq_qr_r(h, A, b, m, n, s, "f64", "f64", "f64", "f64", 1e-10, WL["seed"], {"Y_in": Yfull}, R64, xs64)
        e0.record(stream)
        lsq.lsq_qr_r(h, A, b, m, n, s, "f64", "f64", "f64", "f64", 1e-10, WL["seed"], {"Y_in": Yfull}, R64, xs64)
        e1.record(stream)
        torch.cuda.synchronize()
        qr64 = e0.elapsed_time(e1)
        tol64 = 1e-10
        o64 = {"R_in": R64, "x0_in": xs64}
        lsq.lsq_lsqr(h, A, b, m, n, s, "f64", "f64", "f64", "f64", tol64, WL["seed"], o64, x64)
        e0.record(stream)
        st64, info64 = lsq.lsq_lsqr(h, A, b, m, n, s, "f64", "f64", "f64", "f64", tol64, WL["seed"], o64, x64)
        e1.record(stream)
        torch.cuda.synchronize()
        ls64 = e0.elapsed_time(e1)
        fx64 = (torch.linalg.norm(x64 - x_true) / torch.linalg.norm(x_true)).item()
        fp64 = {"tts_ms": sk64 + qr64 + ls64, "sketch_ms": sk64, "qr_ms": qr64, "lsqr_ms": ls64,
                "lsqr_its": info64.lsqr_its, "lsqr_tol": tol64, "status": st64, "fe_x": fx64,
                "meets_bound": bool(fx64 <= 4 * 2.0 ** -24), "speedup_of_mixed": (sk64 + qr64 + ls64) / value,
                "how": (f"FP64 sketch on CUDA cores timed on the first m/{frac} rows and scaled by {frac} "
                        "(its work is linear in m: extrapolated); FP64 QR and FP64 LSQR timed at full size "
                        "(the QR on the mixed sketch's Y: its cost does not depend on the values, and LSQR "
                        "runs with that R)")}
        del Yfull, Ys, R64, xs64, x64
    except Exception as exc:   # reported, never fatal for the headline line
        fp64 = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- end to end through the C ABI with host buffers (lsq_lsir_host: copies of A and b
    # in, x and r out, inside the timed region), checked bit for bit against the
    # device-pointer solve above
    e2e = {"value": None, "unit": "ms", "h2d_bytes_per_step": int(8 * m * n + 8 * m),
           "d2h_bytes_per_step": int(8 * n + 8 * m), "path": "lsq_lsir_host (host A, b in; host x, r out)"}
    try:
        hA = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        hA.copy_(A)
        hb = torch.empty(m, dtype=torch.float64, pin_memory=True)
        hb.copy_(b)
        hx = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hr = torch.empty(m, dtype=torch.float64, pin_memory=True)
        us = WL["u_s"]

        def host_call():
            return lsq.lsq_lsir_host(h, hA, hb, m, n, s, us, *rest, None, hx, hr)

        host_call()                                   # workspace and graphs for its buffers
        torch.cuda.synchronize()
        e2e["bit_equal_to_device_solve"] = bool(torch.equal(hx, x.cpu()) and torch.equal(hr, r.cpu()))
        k_e2e = max(1, min(3, args.steps))
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(k_e2e):
            host_call()
        e3.record(stream)
        torch.cuda.synchronize()
        e2e["value"] = barrier_max(e2.elapsed_time(e3) / k_e2e, world) / world
        del hA, hb, hx, hr
    except Exception as exc:                          # recorded in the line, never fatal
        e2e["error"] = f"{type(exc).__name__}: {exc}"

    # ---- the secondary configuration (m = 1e5, n = 500, kappa = 1e6), device-drawn
    secondary = None
    del A, b
    torch.cuda.empty_cache()
    try:
        g2 = DeviceRandsvd(WL2["m"], WL2["n"], seed=WL2["data_seed"])
        A2, b2, rp2 = g2.problem(WL2["kappa"], WL2["rho"])
        xt2 = g2.x_true.clone()
        g2.release()
        x2 = torch.zeros(WL2["n"], dtype=torch.float64, device="cuda")
        r2 = torch.zeros(WL2["m"], dtype=torch.float64, device="cuda")
        rest2 = (WL2["u_p"], WL2["u_w"], WL2["u_r"], WL2["tol"], WL2["seed"])
        kw2 = dict(AA=A2, bb=b2, xx=x2, rr=r2, us=WL2["u_s"], mm=WL2["m"], nn=WL2["n"], ss=WL2["s"], rst=rest2)
        for _ in range(3):
            solve(None, **kw2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k2 = 10
        e0.record(stream)
        for _ in range(k2):
            st2, i2 = solve(None, **kw2)
        e1.record(stream)
        torch.cuda.synchronize()
        d2 = i2.as_dict()
        fx2, fr2 = fe(x2, r2, xt2, rp2)
        secondary = {"config": WL2, "ms_per_solve": e0.elapsed_time(e1) / k2, "converged": bool(d2["ir_converged"]),
                     "iterations": {"lsqr": d2["lsqr_its"], "ir": d2["ir_its"], "fgmres_total": d2["gmres_its_total"]},
                     "fe_x": fx2, "fe_r": fr2, "meets_bound": bool(max(fx2, fr2) <= 4 * 2.0 ** -24),
                     "stage_ms": d2["stage_ms"]}
        del A2, b2, x2, r2
    except Exception as exc:
        secondary = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- batched configuration: 512 uneven problems in one grouped call (the headline
    # handle's workspace -- tens of GB at m = 4e6 -- is released first)
    h.close()
    torch.cuda.empty_cache()
    batched = None
    if rank == 0 and not args.no_batched:
        try:
            batched = run_batched(lsq, torch, pk, fp64_fma)
        except Exception as e:   # reported, never fatal for the headline line
            batched = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()

    u = 2.0 ** -24
    line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/f32/f64", "data": "synthetic",
            "config": config(),
            "converged": bool(last["ir_converged"]),
            "forward_error": {"x": fe_mixed[0], "r": fe_mixed[1], "bound_4u": 4 * u,
                              "against": "the generator's x and r_perp (stand-ins for the stored-data "
                                         "solution: ~1e-9 apart at kappa=1e7, rho=1e-6)"},
            "mixed_meets_bound": bool(max(fe_mixed) <= 4 * u),
            "iterations": {"lsqr": last["lsqr_its"], "ir": last["ir_its"],
                           "fgmres_total": last["gmres_its_total"], "escalated": last["escalated"]},
            "ir_hist": {"dx_rel": last["ir_dx_hist"], "dr_rel": last["ir_dr_hist"],
                        "gmres_its": last["gmres_its"], "gmres_relres": last["gmres_relres"]},
            "stage_ms": last["stage_ms"], "kappa_R_est": last["kappa_R_est"],
            "kernels": kernels, "roofline": roofline, "tts_roofline": tts_roof,
            "fp64_fma_per_s": fp64_fma,
            "fp64_path": fp64, "single_term_sketch": single, "sparse_sign_sketch": sparse_leg,
            "secondary": secondary, "batched": batched,
            "gpu_launches": int(sum(i["gpu_launches"] for i in infos)),
            "clocks": clocks, "e2e": e2e, "draw_s": t_draw}

    # ---- oracle leg (rank 0, N = 1): the CPU baseline on a bounded sample
    if rank == 0 and world == 1:
        iters = {"lsqr": last["lsqr_its"], "fgmres": last["gmres_its_total"]}
        S = oracle_sample()
        v, detail = oracle_step(S, iters)
        line["cpu_baseline"] = {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                "threads": THREADS_NOTE, "sample": sample_note(iters), "detail": detail}
    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- single cases for profilers
CASES = ("lsir_m4e6", "fgmres_pass_m2e5_n1000", "arnoldi_m1e6_n1000", "arnoldi_m1e6_n200", "sketch_m2e5_n1000",
         "batched_512", "batched_64", "batched_16")


def run_case(name):
    """One untimed call of a small named workload (for ncu captures); prints one status line.

    lsir_m4e6: one lsq_lsir of the bench workload.  fgmres_pass_m2e5_n1000: one
    refinement step (six FGMRES iterations, CUDA graphs off) on a 200000 x 1000
    Gaussian A.  arnoldi_m1e6_n1000: one refinement step of up to 40 FGMRES
    iterations on a 1e6 x 1000, kappa = 1e7 problem (arnoldi_m1e6_n200: the same on a
    1e6 x 200 problem, 2.4 GB on the device).  sketch_m2e5_n1000: one
    lsq_sketch (s = 4000, BF16X3) of a 200000 x 1000 Gaussian A.  batched_512: the batched
    configuration (512 problems, one warm-up and one timed grouped call); batched_64: its
    first 64 problems (and the per-problem mode on them); batched_16: its first 16 problems,
    one grouped call (for launch lists).
    """
    import torch
    import paper_2410_06319_gb300 as lsq
    from lsq_synth.device import DeviceRandsvd
    torch.manual_seed(0)
    if name.startswith("batched_"):
        # the batched configuration (batched_512), or its first 64 problems (batched_64,
        # also timed in the per-problem mode for comparison)
        if name in ("batched_64", "batched_16"):
            BATCH["count"] = int(name.split("_")[1])
        res = run_batched(lsq, torch, peaks(), lsq.lsq_probe_fma_rate("f64"), warm=(name != "batched_16"))
        if name == "batched_64":
            res["per_problem_mode"] = run_batched(lsq, torch, peaks(), lsq.lsq_probe_fma_rate("f64"),
                                                  opts={"batch_mode": 1})
        print(json.dumps({"case": name, **res}), flush=True)
        return
    h = lsq.Handle()

    def randn(m, n):
        return (torch.randn(m, n, dtype=torch.float64, device="cuda"),
                torch.randn(m, dtype=torch.float64, device="cuda"))

    if name in ("lsir_m4e6", "arnoldi_m1e6_n1000", "arnoldi_m1e6_n200"):
        m = WL["m"] if name == "lsir_m4e6" else 1_000_000
        n = 200 if name == "arnoldi_m1e6_n200" else WL["n"]
        s = 4 * n
        gen = DeviceRandsvd(m, n, seed=WL["data_seed"])
        A, b, _ = gen.problem(WL["kappa"], WL["rho"])
        gen.release()
        opts = None if name == "lsir_m4e6" else {"no_graph": 1, "ir_maxit": 1, "gmres_maxit": 40}
    elif name == "fgmres_pass_m2e5_n1000":
        m, n, s = 200_000, 1000, 4000
        A, b = randn(m, n)
        opts = {"no_graph": 1, "ir_maxit": 1, "gmres_maxit": 6, "lsqr_maxit": 3}
    else:
        m, n, s = 200_000, 1000, 4000
        A, b = randn(m, n)
        Y = torch.zeros(s * (n + 1), dtype=torch.float64, device="cuda")
        st = lsq.lsq_sketch(h, A, b, m, n, s, "bf16x3", "f64", "f32", "f64", 1e-6, 0, None, Y)
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "status": st}), flush=True)
        return
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    st, info = lsq.lsq_lsir(h, A, b, m, n, s, WL["u_s"], WL["u_p"], WL["u_w"], WL["u_r"], WL["tol"],
                            WL["seed"], opts, x, r)
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "status": st, "lsqr_its": info.lsqr_its, "ir_its": info.ir_its,
                      "fgmres_its": info.gmres_its_total, "launches": info.gpu_launches}), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batched", action="store_true",
                    help="leave out the batched configuration (512 problems) from the bench line")
    ap.add_argument("--case", default=None, choices=CASES,
                    help="run one small named workload once (no timing; for profilers)")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
