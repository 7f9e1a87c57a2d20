"""QR, LSQR and LSIR through the C ABI against the oracle (Algorithms 1-2)."""
import numpy as np
import pytest
import torch

from conftest import colmajor, dev, from_colmajor
from lsq_synth import paper_problem, randsvd_problem
from oracle import exact, lsir, lsqr, qr, rng, sketch

pytestmark = pytest.mark.gpu


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("up", ["f64", "f32"])
@pytest.mark.parametrize("m,n,s,kappa", [(3000, 50, 200, 10.0), (5000, 130, 400, 1e2), (900, 1, 4, 1.0),
                                         (4000, 257, 600, 1e3)])
def test_qr_parity(lsq, handle, up, m, n, s, kappa):
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=n)
    Y = sketch.sketch(P.A, P.b, s, 2, "f64")
    dt = np.float64 if up == "f64" else np.float32
    R_or, c_or = qr.householder_qr(Y, n, dtype=dt)
    xs_or = qr.sketch_and_solve(R_or, c_or)
    R, xs = zeros(n * n), zeros(n)
    lsq.lsq_qr_r(handle, dev(P.A), dev(P.b), m, n, s, "f64", up, "f32", "f64", 1e-6, 2,
                 {"Y_in": dev(colmajor(Y))}, R, xs)
    Rg = from_colmajor(R, n, n)
    u = 2.0 ** -53 if up == "f64" else 2.0 ** -24
    nR = np.linalg.norm(R_or, 2)
    assert np.allclose(np.tril(Rg, -1), 0)
    assert np.all(np.diag(Rg) >= 0)
    # both are Householder R factors of the same Y: they agree to ~ kappa u
    assert np.linalg.norm(Rg - R_or, 2) <= 20 * n * kappa * u * nR
    # backward error of the GPU factor itself
    Yn = Y[:, :n]
    assert np.linalg.norm(Rg.T @ Rg - Yn.T @ Yn, 2) <= 10 * s * n * u * np.linalg.norm(Yn, 2) ** 2
    xs_ref = np.linalg.lstsq(Yn, Y[:, n], rcond=None)[0]
    assert np.linalg.norm(xs.cpu().numpy() - xs_ref) <= 20 * n * kappa * u * np.linalg.norm(xs_ref) + 1e-300
    assert np.linalg.norm(xs.cpu().numpy() - xs_or) <= 20 * n * kappa * u * np.linalg.norm(xs_or) + 1e-300


def _oracle_fp64(P, s, seed, tol, maxit):
    Y = sketch.sketch(P.A, P.b, s, seed, "f64")
    R, c = qr.householder_qr(Y, P.n)
    x, info = lsqr.lsqr(P.A, P.b, R, qr.sketch_and_solve(R, c), tol, maxit)
    return x, info


def test_all_fp64_path_config0(lsq, handle):
    """Plain method, all FP64 (m=2000, n=50, kappa=1e3, ||r_perp||/||b|| = 1e-4, s=4n, tol 1e-14)."""
    m, n, s = 2000, 50, 200
    P = randsvd_problem(m, n, 1e3, rho=1e-4, seed=0)
    x_or, info_or = _oracle_fp64(P, s, 0, 1e-14, 2 * n)
    x = zeros(n)
    st, info = lsq.lsq_lsqr(handle, dev(P.A), dev(P.b), m, n, s, "f64", "f64", "f64", "f64", 1e-14, 0,
                            None, x)
    xg = x.cpu().numpy()
    assert st == 0
    assert np.linalg.norm(xg - x_or) / np.linalg.norm(x_or) <= 1e-12 * P.kappa
    xstar, _ = exact.reference_solution(P.A, P.b)
    assert np.linalg.norm(xg - xstar) / np.linalg.norm(xstar) <= 1e-12 * P.kappa
    assert abs(info.lsqr_its - info_or["its"]) <= 2
    assert info.gpu_launches > 0


@pytest.mark.parametrize("m,n,kappa", [(3000, 60, 1e2), (2500, 130, 1e4), (800, 1, 1.0)])
def test_fp32_lsqr_with_oracle_preconditioner(lsq, handle, m, n, kappa):
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=3)
    s = 4 * n if n > 1 else 4
    Y = sketch.sketch(P.A, P.b, s, 1, "f32")
    R, c = qr.householder_qr(Y, n, dtype=np.float32)
    xs = qr.sketch_and_solve(R, c)
    x_or, info_or = lsqr.lsqr(P.A, P.b, R, xs, 1e-6, 2 * n, dtype=np.float32)
    x = zeros(n)
    st, info = lsq.lsq_lsqr(handle, dev(P.A), dev(P.b), m, n, s, "f32", "f32", "f32", "f64", 1e-6, 1,
                            {"R_in": dev(colmajor(R)), "x0_in": dev(xs)}, x)
    xstar, _ = exact.reference_solution(P.A, P.b)
    fe_or = np.linalg.norm(x_or - xstar) / np.linalg.norm(xstar)
    fe = np.linalg.norm(x.cpu().numpy() - xstar) / np.linalg.norm(xstar)
    assert fe <= 10 * fe_or + 10 * 2.0 ** -24 * kappa
    assert abs(info.lsqr_its - info_or["its"]) <= 3, (info.lsqr_its, info_or["its"])


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_lsir_mixed_reaches_working_precision(lsq, handle, fmt):
    """Table 3 setting (u single, u_r double) at kappa = 1e2: forward errors <= 4u."""
    P = paper_problem(1e2, seed=0)
    m, n, s = 1000, 100, 400
    xstar, rstar = exact.reference_solution(P.A, P.b)
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, fmt, "f32", "f32", "f64", 1e-6, 0,
                            None, x, r)
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
    assert st == 0 and info.ir_converged == 1
    assert ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (ex, er)
    assert 1 <= info.ir_its <= 3
    assert abs(info.lsqr_its - 16) <= 3           # Table 1: 16 LSQR iterations
    assert 30 <= info.gmres_its[0] <= 50          # Table 3: 39 FGMRES iterations in the first step
    # the oracle run with the same precisions agrees on the outcome
    Y = sketch.sketch(P.A, P.b, s, 0, fmt)
    R, c = qr.householder_qr(Y, n, dtype=np.float32)
    xo, ro, io = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -24, 1e-6, w_dtype=np.float32)
    assert io["converged"]
    assert abs(io["its"] - info.ir_its) <= 1


def test_lsir_full_size_single_term_bf16_flags_condition(lsq, handle):
    """m=1e5, n=500, kappa=1e6: single-term BF16 has kappa(A) u_s >> 1 (Sec. 3.4)."""
    m, n, s = 100000, 500, 2000
    P = randsvd_problem(m, n, 1e6, rho=1e-3, seed=1)
    A, b = dev(P.A), dev(P.b)
    # warning bit, still finite iterates
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, A, b, m, n, s, "bf16", "f32", "f32", "f64", 1e-6, 0,
                            {"ir_maxit": 2}, x, r)
    assert st in (0, 1) and (info.flags & 1)
    assert np.all(np.isfinite(x.cpu().numpy()))


def test_lsir_full_size_bench_workload(lsq, handle):
    """m=1e5, n=500, kappa=1e6, rho=1e-3, s=4n, BF16X3 sketch, FP32 QR/LSQR, FP64 residuals
    (the bench workload)."""
    m, n, s = 100000, 500, 2000
    P = randsvd_problem(m, n, 1e6, rho=1e-3, seed=1)
    A, b = dev(P.A), dev(P.b)
    # the three-term split sketch: converges to the working-precision level
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, A, b, m, n, s, "bf16x3", "f32", "f32", "f64", 1e-6, 0, None, x, r)
    assert st == 0 and info.ir_converged == 1
    xg, rg = x.cpu().numpy(), r.cpu().numpy()
    xstar, rstar = exact.reference_solution(P.A, P.b, maxit=3)
    ex, er = exact.forward_errors(xg, rg, xstar, rstar)
    assert ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (ex, er)


def test_escalation_rule(lsq, handle):
    """Sec. 5: a non-converged refinement is re-run with FP64 FGMRES products iff kappa < 1/u_s."""
    P = paper_problem(1e2, seed=1)
    m, n, s = 1000, 100, 400
    x, r = zeros(n), zeros(m)
    base = {"ir_maxit": 1, "gmres_maxit": 2}
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "f16", "f32", "f32", "f64", 1e-6, 0,
                            dict(base, kappa_hint=10.0), x, r)
    assert info.escalated == 1 and (info.flags & 2)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "f16", "f32", "f32", "f64", 1e-6, 0,
                            dict(base, kappa_hint=1e5), x, r)
    assert info.escalated == 0 and st == 1
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "f16", "f32", "f32", "f64", 1e-6, 0,
                            dict(base, kappa_hint=10.0, no_escalate=1), x, r)
    assert info.escalated == 0


@pytest.mark.parametrize("n", [101, 37])
def test_fp64_refinement_with_odd_row_stride(lsq, handle, n):
    """FP64 FGMRES products (Sec. 5's escalation, and u = FP64) on an A whose rows
    are not a multiple of 16 bytes: the solve runs on a padded copy."""
    m, s, kappa = 2000, 4 * n, 1e2
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=n)
    xe, re = exact.reference_solution(P.A, P.b)
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "f16", "f32", "f32", "f64", 1e-6, 0,
                            {"ir_maxit": 1, "gmres_maxit": 2, "kappa_hint": 10.0}, x, r)
    assert info.escalated == 1
    assert np.linalg.norm(x.cpu().numpy() - xe) <= 1e-6 * np.linalg.norm(xe)
    # u = u_r = FP64: the residual is no more accurate than the working precision,
    # so the corrections stall at the rounding level and the ||d|| <= u rule does
    # not fire (the oracle with plain FP64 residuals does the same); the forward
    # errors still reach the level of the oracle's
    its = 3
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "bf16", "f64", "f64", "f64", 1e-15, 0,
                            {"ir_maxit": its}, x, r)
    Y = sketch.sketch(P.A, P.b, s, 0, "bf16")
    R, c = qr.householder_qr(Y, n)
    xo, ro, io = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -53, 1e-15, ir_maxit=its,
                           w_dtype=np.float64, ur="f64")
    assert st == (0 if io["converged"] else 1) and info.ir_its == io["its"]
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xe, re)
    exo, ero = exact.forward_errors(xo, ro, xe, re)
    assert ex <= max(10 * exo, 1e-14) and er <= max(10 * ero, 1e-12), (ex, er, exo, ero)


@pytest.mark.parametrize("n", [1000, 901])
def test_fp64_products_on_rows_wider_than_the_bulk_ring(lsq, handle, n):
    """FP64 rows of more than 800 columns (n = 1000 in the largest configurations) do not
    fit two stages of the bulk-streamed ring: the residual pass, the escalated FGMRES
    products and the all-FP64 LSQR run on the register-blocked pass instead."""
    m, s, kappa = 6000, 4 * n, 1e2
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=n)
    xt = P.x_true                      # the stored-data solution is within ~1e-14 of it here
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "f16", "f32", "f32", "f64", 1e-6, 0,
                            {"ir_maxit": 1, "gmres_maxit": 2, "kappa_hint": 10.0}, x, r)
    assert info.escalated == 1
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-6 * np.linalg.norm(xt)
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "bf16x3", "f32", "f32", "f64", 1e-6, 0,
                            None, x, r)
    rp = P.b - P.A @ xt
    ex = np.linalg.norm(x.cpu().numpy() - xt) / np.linalg.norm(xt)
    er = np.linalg.norm(r.cpu().numpy() - rp) / np.linalg.norm(rp)
    assert st == 0 and ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (ex, er)
    x = zeros(n)
    st, info = lsq.lsq_lsqr(handle, dev(P.A), dev(P.b), m, n, s, "f64", "f64", "f64", "f64", 1e-14, 0,
                            None, x)
    assert st == 0 and np.linalg.norm(x.cpu().numpy() - xt) <= 1e-12 * kappa * np.linalg.norm(xt)


def test_invalid_and_degenerate_inputs(lsq, handle):
    P = randsvd_problem(300, 5, 10.0, seed=2)
    x = zeros(5)
    A, b = dev(P.A), dev(P.b)
    bad = [(300, 5, 4, 1e-6), (4, 5, 5, 1e-6), (300, 5, 301, 1e-6), (300, 5, 20, 0.0),
           (300, 5, 20, float("nan")), (300, 2000, 2000, 1e-6)]
    for m, n, s, tol in bad:
        with pytest.raises(lsq.LsqError) as e:
            lsq.lsq_lsqr(handle, A, b, m, n, s, "bf16", "f32", "f32", "f64", tol, 0, None, x)
        assert e.value.status == -1
    with pytest.raises(lsq.LsqError):
        lsq.lsq_lsqr(handle, A, b, 300, 5, 20, "bf16", "f32", "f32", "f32", 1e-6, 0, None, x)
    # a zero column makes R singular -> LSQ_E_RANK
    Az = P.A.copy()
    Az[:, 2] = 0.0
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_lsqr(handle, dev(Az), b, 300, 5, 20, "f64", "f64", "f64", "f64", 1e-10, 0, None, x)
    assert e.value.status == -2
    # b = 0: the least-squares solution is 0
    st, info = lsq.lsq_lsqr(handle, A, dev(np.zeros(300)), 300, 5, 20, "f64", "f64", "f64", "f64",
                            1e-12, 0, None, x)
    assert np.all(x.cpu().numpy() == 0.0)


def test_deterministic_and_timing_instrumentation(lsq, handle):
    """Repeated calls (cached CUDA graphs) give bit-identical results; timing adds no drift."""
    P = randsvd_problem(6000, 96, 1e3, rho=1e-2, seed=9)
    m, n, s = 6000, 96, 384
    outs = []
    for opts in (None, None, {"timing": 1}):
        x, r = zeros(n), zeros(m)
        st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "bf16", "f32", "f32", "f64", 1e-6,
                                3, opts, x, r)
        outs.append((x.cpu().numpy(), r.cpu().numpy(), info.as_dict()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[2][0])
    d = outs[2][2]
    assert d["kern_launches"]["lsqr_pass"] == d["lsqr_its"]
    assert d["kern_launches"]["fgmres_pass"] == d["gmres_its_total"]
    assert d["kern_launches"]["arnoldi_step"] == d["gmres_its_total"]
    assert d["kern_launches"]["fgmres_trsv"] == 2 * d["gmres_its_total"]
    assert d["kern_launches"]["residual_pass"] == d["ir_its"]
    assert d["kern_launches"]["sketch_gemm"] == 1
    assert all(v > 0 for k, v in d["kern_ms"].items() if not k.startswith("spare"))
    assert outs[0][2]["kern_launches"]["lsqr_pass"] == 0


def test_lsir_split_sketch_converges_where_bf16_fails(lsq, handle):
    """kappa(A) = 1e6: BF16 breaks kappa u_s < 1 (Sec. 3.4), the three-term split restores it."""
    P = paper_problem(1e6, seed=3)
    m, n, s = 1000, 100, 400
    xstar, rstar = exact.reference_solution(P.A, P.b)
    out = {}
    for fmt in ("bf16", "bf16x3"):
        x, r = zeros(n), zeros(m)
        st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, fmt, "f32", "f32", "f64", 1e-6, 0,
                                None, x, r)
        out[fmt] = (st, info.as_dict(), exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar))
    st, info, (ex, er) = out["bf16x3"]
    assert st == 0 and ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (ex, er, info)
    assert not (info["flags"] & 1)                        # kappa_est u_s < 1: no warning
    assert info["lsqr_its"] <= 25
    st_b, info_b, _ = out["bf16"]
    assert info_b["flags"] & 1                            # kappa u_s >= 1 flagged
    assert info_b["lsqr_its"] > 2 * info["lsqr_its"]      # weaker preconditioner (Table 1)
    # the oracle agrees on the split sketch's quality
    Y = sketch.sketch(P.A, P.b, s, 0, "bf16x3")
    R, c = qr.householder_qr(Y, n, dtype=np.float32)
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    assert sv[0] / sv[-1] < 4.0


def test_batched_uneven_problems_match_single_solves(lsq, handle):
    """lsq_lsir_batched in per-problem mode over uneven problems equals lsq_lsir on each problem."""
    shapes = [(3000, 32, 1e2), (7000, 64, 1e4), (5000, 100, 1e3), (4100, 45, 10.0), (9000, 77, 1e5)]
    probs, singles, P_all = [], [], []
    for k, (m, n, kappa) in enumerate(shapes):
        P = randsvd_problem(m, n, kappa, rho=1e-3, seed=40 + k)
        P_all.append(P)
        A, b = dev(P.A), dev(P.b)
        x, r = zeros(n), zeros(m)
        probs.append(dict(A=A, b=b, m=m, n=n, s=4 * n, seed=k, x=x, r=r))
        xs, rs = zeros(n), zeros(m)
        lsq.lsq_lsir(handle, A, b, m, n, 4 * n, "bf16x3", "f32", "f32", "f64", 1e-6, k, None, xs, rs)
        singles.append((xs.cpu().numpy(), rs.cpu().numpy()))
    st, sts, infos = lsq.lsq_lsir_batched(handle, probs, "bf16x3", "f32", "f32", "f64", 1e-6, {"batch_mode": 1})
    assert st == 0 and all(v == 0 for v in sts)
    for k, pr in enumerate(probs):
        assert np.array_equal(pr["x"].cpu().numpy(), singles[k][0])
        assert np.array_equal(pr["r"].cpu().numpy(), singles[k][1])
        assert infos[k].ir_converged == 1


def test_auto_sketch_precision_follows_the_condition(lsq, handle):
    """LSQ_AUTO (Sec. 3.4, Sec. 6: u_s kappa(A) < 1 with kappa(A) estimated from R): BF16 where
    kappa(A) u_s is small, the single-precision split where BF16 is regularised; both reach
    the 4u level (Table 3 setting)."""
    out = {}
    for kappa in (10.0, 1e6):
        P = paper_problem(kappa, seed=7)
        m, n, s = 1000, 100, 400
        x, r = zeros(n), zeros(m)
        st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "auto", "f32", "f32", "f64", 1e-6, 0,
                                None, x, r)
        xstar, rstar = exact.reference_solution(P.A, P.b)
        ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
        out[kappa] = (info.us_used, info.sketches)
        assert st == 0 and ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (kappa, ex, er, out[kappa])
    assert out[10.0] == (lsq.PREC["bf16"], 1), out
    assert out[1e6] == (lsq.PREC["bf16x3"], 2), out
    # the choice needs the QR that follows the sketch
    Y = zeros(400 * 101)
    P = paper_problem(10.0, seed=7)
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_sketch(handle, dev(P.A), dev(P.b), 1000, 100, 400, "auto", "f32", "f32", "f64", 1e-6, 0, None, Y)
    assert e.value.status == -1
