"""Pins for the oracle's Algorithm 1: the sketch and its Householder R."""
import numpy as np
import pytest

from lsq_synth import randsvd_problem, paper_problem
from oracle import lsqr, qr, rng, sketch, theory


def _explicit_omega(s, m, seed, fmt="f64"):
    return rng.round_to_format(rng.gaussian_block(0, s, 0, m, seed), fmt) / np.sqrt(s)


def test_column_scale_puts_column_max_in_target_binade():
    r = np.random.default_rng(0)
    M = r.standard_normal((50, 7)) * np.array([1e-30, 1e-5, 1, 3, 1e5, 1e20, 0.0])
    for fmt, t in (("f16", 14), ("bf16", 14), ("e4m3", 7)):
        k = sketch.column_scale_exponents(M, fmt)
        cm = np.abs(np.ldexp(M, k[None, :])).max(axis=0)
        assert np.all((cm[:-1] >= 2.0 ** t) & (cm[:-1] < 2.0 ** (t + 1)))
        assert k[-1] == 0                       # an all-zero column is left alone
    assert np.all(sketch.column_scale_exponents(M, "f32") == 0)


def test_sketch_f64_is_omega_times_data():
    P = randsvd_problem(300, 6, 1e3, seed=1)
    Y = sketch.sketch(P.A, P.b, 24, 5, "f64")
    Om = _explicit_omega(24, 300, 5)
    ref = Om @ np.column_stack([P.A, P.b])
    assert np.allclose(Y, ref, rtol=0, atol=1e-13 * (np.abs(Om) @ np.abs(np.column_stack([P.A, P.b]))).max())


def test_sketch_cast_error_within_paper_model():
    """Sec. 3.2: ||Delta_s|| <= u_s ||A|| ||Omega|| (+ product term, here FP64 and negligible)."""
    P = randsvd_problem(2000, 20, 1e2, seed=2)
    Y64 = sketch.sketch(P.A, P.b, 80, 1, "f64")
    for fmt in ("bf16", "f16", "e4m3"):
        Ys = sketch.sketch(P.A, P.b, 80, 1, fmt)
        Om = _explicit_omega(80, 2000, 1, fmt)
        Ab = np.column_stack([P.A, P.b])
        # the rounded Omega is a fixed sketch; the cast of A is the error term
        ref = Om @ Ab
        err = np.linalg.norm(Ys - ref, 2)
        us = rng.UNIT_ROUNDOFF[fmt]
        bound = us * np.linalg.norm(Ab, 2) * np.linalg.norm(Om, 2) * np.sqrt(Ab.shape[1])
        assert err <= bound
        assert err > 0
        assert np.linalg.norm(Y64 - Ys, 2) > 0


def test_sketch_preserves_norms_in_expectation():
    r = np.random.default_rng(3)
    x = r.standard_normal((4000, 1))
    vals = []
    for seed in range(40):
        y = sketch.sketch(x, np.zeros(4000), 32, seed, "f64")[:, 0]
        vals.append(np.dot(y, y) / np.dot(x[:, 0], x[:, 0]))
    vals = np.array(vals)
    # E ||Omega x||^2 = ||x||^2; Var = 2/s per draw
    assert abs(vals.mean() - 1) < 4 * np.sqrt(2 / 32 / len(vals))


def test_householder_r_matches_lapack_up_to_row_signs():
    r = np.random.default_rng(4)
    Y = r.standard_normal((60, 9))
    R, c = qr.householder_qr(Y, 8)
    Rl = np.linalg.qr(Y[:, :8], mode="r")
    Rl = Rl * np.where(np.diag(Rl) < 0, -1.0, 1.0)[:, None]
    assert np.allclose(R, Rl, atol=1e-12)
    Q, _ = np.linalg.qr(Y[:, :8])
    cl = (Q.T @ Y[:, 8]) * np.where(np.diag(np.linalg.qr(Y[:, :8], mode="r")) < 0, -1.0, 1.0)
    assert np.allclose(c, cl, atol=1e-12)
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)
    assert np.allclose(R.T @ R, Y[:, :8].T @ Y[:, :8], atol=1e-11)


def test_householder_closed_forms_small_n():
    y = np.array([[3.0, 1.0], [4.0, 2.0]])
    R, c = qr.householder_qr(y, 1)
    assert R.shape == (1, 1) and abs(R[0, 0] - 5.0) < 1e-15     # n = 1: R = ||y||
    assert abs(c[0] - (3 * 1 + 4 * 2) / 5.0) < 1e-15            # q^T b
    Y = np.array([[1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])
    R, _ = qr.householder_qr(Y, 2)
    # Gram-Schmidt by hand: r11 = sqrt2, r12 = 1/sqrt2, r22 = sqrt(3/2)
    assert np.allclose(R, [[np.sqrt(2), 1 / np.sqrt(2)], [0, np.sqrt(1.5)]], atol=1e-15)


def test_householder_float32_backward_error():
    r = np.random.default_rng(6)
    Y = r.standard_normal((200, 40)) @ np.diag(np.logspace(0, -3, 40))
    R, _ = qr.householder_qr(Y, 40, dtype=np.float32)
    err = np.linalg.norm(R.T @ R - Y.T @ Y) / np.linalg.norm(Y) ** 2
    assert err < 200 * 40 * 2.0 ** -24


def test_sketch_and_solve_is_sketched_lstsq():
    P = randsvd_problem(500, 8, 1e2, seed=7)
    Y = sketch.sketch(P.A, P.b, 32, 3, "f64")
    R, c = qr.householder_qr(Y, 8)
    xs = qr.sketch_and_solve(R, c)
    ref = np.linalg.lstsq(Y[:, :8], Y[:, 8], rcond=None)[0]
    assert np.allclose(xs, ref, rtol=1e-12, atol=1e-12 * np.linalg.norm(ref))


def test_preconditioned_kappa_equals_kappa_omega_u():
    """Sec. 2: kappa(A R^-1) = kappa(Omega U), ||A R^-1|| = ||(Omega U)^+|| (exact sketch)."""
    P = randsvd_problem(800, 10, 1e3, seed=8)
    Y = sketch.sketch(P.A, P.b, 40, 9, "f64")
    R, _ = qr.householder_qr(Y, 10)
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    U = np.linalg.svd(P.A, full_matrices=False)[0]
    so = np.linalg.svd(_explicit_omega(40, 800, 9) @ U, compute_uv=False)
    assert abs(sv[0] / sv[-1] - so[0] / so[-1]) < 1e-9 * so[0] / so[-1]
    assert abs(sv[0] - 1 / so[-1]) < 1e-9 * sv[0]
    assert abs(1 / sv[-1] - so[0]) < 1e-9 * so[0]


def test_paper_good_regime_values(golden):
    """Fig. 3(b)/4(c): ||AR^-1|| ~ 2.03, ||(AR^-1)^+|| ~ 1.46, kappa ~ 2.97 (m=1000, n=100, s=4n)."""
    vals = {r[0]: float(r[1]) for r in golden("paper_fig3_good_regime.txt")}
    na, npv, ka = [], [], []
    for seed in range(3):
        P = paper_problem(1e2, seed=seed)
        Y = sketch.sketch(P.A, P.b, 400, seed, "f32")
        R, _ = qr.householder_qr(Y, 100, dtype=np.float32)
        sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
        na.append(sv[0]); npv.append(1 / sv[-1]); ka.append(sv[0] / sv[-1])
    assert abs(np.mean(na) - vals["norm_AR"]) < 0.1 * vals["norm_AR"]
    assert abs(np.mean(npv) - vals["norm_AR_pinv"]) < 0.05 * vals["norm_AR_pinv"]
    assert abs(np.mean(ka) - vals["kappa_AR"]) < 0.1 * vals["kappa_AR"]
    # and the Marchenko-Pastur limits at n/s = 1/4 (2, 1.5, 3) hold to ~10%
    mp = theory.mp_limits(100, 400)
    assert abs(np.mean(ka) - mp[2]) < 0.1 * mp[2]


def test_low_precision_sketch_degrades_as_paper_predicts():
    """Sec. 3.4 / Fig. 3(a): kappa(A) u_s >> 1 makes ||(A R^-1)^+|| grow; << 1 keeps it ~1.5."""
    P = paper_problem(1e6, seed=1)
    out = {}
    for fmt in ("f32", "bf16"):
        Y = sketch.sketch(P.A, P.b, 400, 1, fmt)
        R, _ = qr.householder_qr(Y, 100)
        sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
        out[fmt] = 1 / sv[-1]
    assert out["f32"] < 1.7
    assert out["bf16"] > 20 * out["f32"]
    # Corollary bound of Sec. 3.4: ||(A R_s^-1)^+|| <= (1 + sqrt(n) u_s kappa) ||Omega||
    Om = _explicit_omega(400, 1000, 1, "bf16")
    assert out["bf16"] <= (1 + np.sqrt(100) * 2.0 ** -8 * 1e6) * np.linalg.norm(Om, 2)


def test_split3_carries_single_precision():
    r = np.random.default_rng(11)
    x = r.standard_normal(20000) * np.exp(r.uniform(-20, 20, 20000))
    hi, lo, lo2 = rng.split3(x, "bf16")
    for t in (hi, lo, lo2):
        assert np.array_equal(rng.round_to_format(t, "bf16"), t)      # each term is a BF16 value
    assert np.all(np.abs(x - (hi + lo + lo2)) <= 2.0 ** -24 * np.abs(x))
    assert np.all(np.abs(lo) <= 2.0 ** -8 * np.abs(hi) + 1e-300)


def test_bf16x3_operand_is_the_single_precision_cast():
    """Sec. 3.2 with u_s = single: the BF16X3 operand is fl_single(2^k A), carried exactly by
    three BF16 terms (numpy's own FP32 conversion is the reference).  Entries 2^-130 below
    their column's maximum put the third term on BF16's subnormal grid, the one place the
    terms may miss y (by at most half its spacing, 2^-134)."""
    r = np.random.default_rng(12)
    A = r.standard_normal((3000, 7)) * np.exp(r.uniform(-30, 30, (1, 7)))
    A[::17, 3] *= 2.0 ** -60
    A[::13, 5] *= 2.0 ** -130
    b = r.standard_normal(3000)
    As, bs, kA, kb = sketch.cast_scaled(A, b, "bf16x3")
    y = np.ldexp(A, kA[None, :]).astype(np.float32).astype(np.float64)
    assert np.all(np.abs(As - y) <= 2.0 ** -134)
    deep = np.abs(y) < 2.0 ** -100
    assert deep.sum() > 100 and np.array_equal(As[~deep], y[~deep])
    assert np.array_equal(bs, np.ldexp(b, kb).astype(np.float32).astype(np.float64))
    for t in rng.split3(y, "bf16"):
        assert np.array_equal(rng.round_to_format(t, "bf16"), t)
    # a split of the FP64 entries (no single-precision cast first) is a different operand
    hi, lo, lo2 = rng.split3(np.ldexp(A, kA[None, :]), "bf16")
    assert np.mean((hi + lo + lo2) != y) > 0.2


def test_split_sketch_restores_the_good_regime():
    """Sec. 3.4: with the single-precision split sketch kappa(A R^-1) stays ~3 at kappa(A) = 1e6."""
    P = paper_problem(1e6, seed=2)
    Y = sketch.sketch(P.A, P.b, 400, 2, "bf16x3")
    R, _ = qr.householder_qr(Y, 100)
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    assert sv[0] / sv[-1] < 1.2 * theory.mp_limits(100, 400)[2]
    Yb = sketch.sketch(P.A, P.b, 400, 2, "bf16")
    Rb, _ = qr.householder_qr(Yb, 100)
    svb = np.linalg.svd(P.A @ np.linalg.inv(Rb), compute_uv=False)
    assert svb[0] / svb[-1] > 10 * sv[0] / sv[-1]


def _kappa_AR(A, R):
    sv = np.linalg.svd(np.linalg.solve(np.asarray(R, np.float64).T, A.T).T, compute_uv=False)
    return sv[0] / sv[-1]


def test_sketch_accumulated_in_us_reproduces_fig3(golden):
    """Fig. 3(a), (b), 4(a): with the product formed in u_s (Sec. 3.2's model) the oracle's
    ||A R^-1||, ||(A R^-1)^+||, kappa(A R^-1) and the preconditioned augmented condition
    number (Eq. 4.1) follow the printed values (one draw each: norms within 15 %, condition
    numbers within 25 %); with the product accumulated in FP64 only the cast error is left,
    and kappa(A R^-1) is ten times smaller or more once kappa u_s >> 1 -- the regime the
    FP32-accumulating tensor cores are in."""
    for src, kappa, *vals in golden("paper_half_sketch.txt"):
        if src not in ("fig3a", "fig3b", "fig4a"):
            continue
        fmt = "f32" if src == "fig3b" else "f16"
        kappa = float(kappa)
        kar, kaug, nar, narp = (float(v) for v in vals)
        P = paper_problem(kappa, seed=0)
        Yh = sketch.sketch(P.A, P.b, 400, 0, fmt, accumulate="us")
        Rh, _ = qr.householder_qr(Yh, 100, dtype=np.float64 if src == "fig4a" else np.float32)
        sv = np.linalg.svd(np.linalg.solve(np.asarray(Rh, np.float64).T, P.A.T).T, compute_uv=False)
        ctx = (kappa, sv[0], 1 / sv[-1])
        assert 0.85 * nar <= sv[0] <= 1.15 * nar and 0.85 * narp <= 1 / sv[-1] <= 1.15 * narp, ctx
        assert 0.75 * kar <= sv[0] / sv[-1] <= 1.25 * kar, ctx
        assert 0.75 * kaug <= theory.kappa_prec_aug(1.0, sv[0], sv[-1]) <= 1.25 * kaug, ctx
        if src == "fig3a" and kappa >= 1e5:
            Y64 = sketch.sketch(P.A, P.b, 400, 0, "f16")
            R64, _ = qr.householder_qr(Y64, 100, dtype=np.float32)
            assert _kappa_AR(P.A, R64) <= 0.1 * kar


def test_fig3a_printed_columns_satisfy_eq41(golden):
    """The printed kappa(M_L^-1 Atilde M_R^-1) of Figs. 3-4 is Eq. 4.1 of the printed
    ||A R^-1|| and ||(A R^-1)^+|| in the broken regime too (to the printed digits)."""
    for src, kappa, *vals in golden("paper_half_sketch.txt"):
        if src not in ("fig3a", "fig3b", "fig4a"):
            continue
        kar, kaug, nar, narp = (float(v) for v in vals)
        assert abs(theory.kappa_prec_aug(1.0, nar, 1 / narp) - kaug) <= 0.015 * kaug, (kappa, kaug)


def test_sketch_accumulated_in_us_lsqr_counts_tables_1_2(golden):
    """Tables 1-2: LSQR slows down and hits its cap as kappa u_s grows (u single, tol 1e-6;
    u double, tol 1e-12), with the sketch product formed in u_s."""
    for src, kappa, its, *rest in golden("paper_half_sketch.txt"):
        if src not in ("T1", "T2"):
            continue
        kappa, its = float(kappa), int(its)
        fmt = {"half": "f16", "single": "f32"}[rest[0]]
        dt, tol = (np.float32, 1e-6) if src == "T1" else (np.float64, 1e-12)
        got = []
        for seed in range(2):
            P = paper_problem(kappa, seed=seed)
            Y = sketch.sketch(P.A, P.b, 400, seed, fmt, accumulate="us")
            R, c = qr.householder_qr(Y, 100, dtype=dt)
            _, info = lsqr.lsqr(P.A, P.b, R, qr.sketch_and_solve(R, c), tol, 200, dtype=dt)
            got.append(info["its"])
        assert abs(np.mean(got) - its) <= max(2, 0.2 * its), (src, kappa, got, its)


def test_sketch_accumulated_in_us_lsir_tables_3_4(golden):
    """Tables 3-4: with the sketch product formed in u_s, one refinement step of 45 FGMRES
    iterations for the half sketch at kappa = 1e3 (u single); no convergence in 30 steps,
    and no escalation since kappa >= 1/u_s (Sec. 5), where the tables print "-"."""
    from oracle import exact, lsir
    for src, kappa, *vals in golden("paper_half_sketch.txt"):
        if src not in ("T3", "T4"):
            continue
        steps, gm, prec = vals
        kappa = float(kappa)
        fmt = {"half": "f16", "single": "f32"}[prec]
        dt, u, tol = (np.float32, 2.0 ** -24, 1e-6) if src == "T3" else (np.float64, 2.0 ** -53, 1e-12)
        P = paper_problem(kappa, seed=0)
        xstar, rstar = exact.reference_solution(P.A, P.b)
        Y = sketch.sketch(P.A, P.b, 400, 0, fmt, accumulate="us")
        R, c = qr.householder_qr(Y, 100, dtype=dt)
        x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), u, tol, w_dtype=dt,
                               us=rng.UNIT_ROUNDOFF[fmt], kappa=kappa, xstar=xstar, rstar=rstar)
        if steps == "-":
            assert not info["converged"] and not info["escalated"] and info["its"] == 30, (src, kappa)
        else:
            assert info["converged"] and info["its"] == int(steps)
            assert abs(info["gmres_total"] - int(gm)) <= 3, info
