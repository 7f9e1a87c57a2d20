"""Pins for the oracle's LSQR, FGMRES and LSIR (Algorithm 2)."""
import numpy as np
import pytest

from lsq_synth import paper_problem, randsvd_problem
from oracle import exact, fgmres, lsir, lsqr, qr, rng, sketch, theory


def _precond(P, s, seed=0, fmt="f64"):
    Y = sketch.sketch(P.A, P.b, s, seed, fmt)
    R, c = qr.householder_qr(Y, P.n)
    return R, qr.sketch_and_solve(R, c)


def _krylov_ls(M, rhs, k):
    """argmin_z ||rhs - M z|| over z in K_k(M^T M, M^T rhs), via an explicit basis."""
    q = M.T @ rhs
    K = [q / np.linalg.norm(q)]
    for _ in range(k - 1):
        v = M.T @ (M @ K[-1])
        for u in K:                        # orthogonalise twice
            v -= np.dot(u, v) * u
        for u in K:
            v -= np.dot(u, v) * u
        K.append(v / np.linalg.norm(v))
    B = np.column_stack(K)
    c = np.linalg.lstsq(M @ B, rhs, rcond=None)[0]
    return B @ c


def test_lsqr_iterates_are_krylov_minimisers():
    P = randsvd_problem(200, 12, 1e2, seed=1)
    R, xs = _precond(P, 48)
    Ahat = P.A @ np.linalg.inv(R)
    rbar = P.b - P.A @ xs
    for k in (1, 2, 4, 6):
        x, info = lsqr.lsqr(P.A, P.b, R, xs, 0.0, k)
        assert info["its"] == k
        z_ref = _krylov_ls(Ahat, rbar, k)
        x_ref = xs + np.linalg.solve(R, z_ref)
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
        # phibar is the true residual norm (Paige-Saunders invariant)
        assert abs(info["normr"] - np.linalg.norm(P.b - P.A @ x)) <= 1e-10 * np.linalg.norm(P.b)


def test_lsqr_converges_to_least_squares_solution():
    P = randsvd_problem(400, 10, 1e3, rho=1e-2, seed=2)
    R, xs = _precond(P, 40)
    x, info = lsqr.lsqr(P.A, P.b, R, xs, 1e-14, 40)
    xstar, _ = exact.reference_solution(P.A, P.b)
    assert info["flag"] in (1, 2)
    assert np.linalg.norm(x - xstar) / np.linalg.norm(xstar) < 1e-12 * P.kappa
    # the normal equations hold: A^T (b - A x) ~ 0
    g = P.A.T @ exact.residual(P.A, P.b, x)
    assert np.linalg.norm(g) < 1e-12 * np.linalg.norm(P.A, 2) * np.linalg.norm(P.b)


def test_lsqr_small_case_against_extended_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    P = randsvd_problem(30, 5, 1e4, rho=1e-1, seed=3)
    R, xs = _precond(P, 20)
    x, _ = lsqr.lsqr(P.A, P.b, R, xs, 1e-15, 30)
    A = mp.matrix(P.A.tolist())
    b = mp.matrix(P.b.tolist())
    xe = mp.lu_solve(A.T * A, A.T * b)
    xe = np.array([float(v) for v in xe])
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) < 1e-16 * P.kappa ** 2 * 10


def test_lsqr_iteration_counts_match_paper_tables(golden):
    rows = [r for r in golden("paper_tables.txt") if r[0] in ("T1", "T2")]
    for table, kappa, us, u, its, _, _ in rows:
        kappa = float(kappa)
        fmt = {"half": "f16", "single": "f32", "double": "f64"}[us]
        dt = np.float32 if u == "single" else np.float64
        tol = 1e-6 if u == "single" else 1e-12
        got = []
        for seed in range(2):
            P = paper_problem(kappa, seed=seed)
            Y = sketch.sketch(P.A, P.b, 400, seed, fmt)
            R, c = qr.householder_qr(Y, 100, dtype=dt)
            x, info = lsqr.lsqr(P.A, P.b, R, qr.sketch_and_solve(R, c), tol, 200, dtype=dt)
            got.append(info["its"])
        assert abs(np.mean(got) - int(its)) <= 2, (table, kappa, us, got, its)


def test_lsqr_forward_errors_match_paper_tables(golden):
    """Tables 1-2 print LSQR's forward errors against x*, r*.  The oracle's (geometric
    mean over three draws of the recipe) lie within a factor 2 of them for kappa <= 1e2
    and within 8 beyond, where one realisation's error varies more with kappa."""
    for table, kappa, us, u, px, pr in golden("paper_lsqr_errors.txt"):
        kappa, px, pr = float(kappa), float(px), float(pr)
        fmt = {"single": "f32", "double": "f64"}[us]
        dt = np.float32 if u == "single" else np.float64
        tol = 1e-6 if u == "single" else 1e-12
        errs = []
        for seed in range(3):
            P = paper_problem(kappa, seed=seed)
            xstar, rstar = exact.reference_solution(P.A, P.b)
            Y = sketch.sketch(P.A, P.b, 400, seed, fmt)
            R, c = qr.householder_qr(Y, 100, dtype=dt)
            x, _ = lsqr.lsqr(P.A, P.b, R, qr.sketch_and_solve(R, c), tol, 200, dtype=dt)
            errs.append(exact.forward_errors(x, P.b - P.A @ x, xstar, rstar))
        gx, gr = np.exp(np.mean(np.log(errs), axis=0))
        f = 2.0 if kappa <= 1e2 else 8.0
        assert px / f <= gx <= px * f and pr / f <= gr <= pr * f, (table, kappa, gx, gr, px, pr)


def _dense_aug_prec(A, R):
    m, n = A.shape
    Ri = np.linalg.inv(R)
    ML = np.block([[np.eye(m), np.zeros((m, n))], [np.zeros((n, m)), Ri.T]])
    MR = np.block([[np.eye(m), np.zeros((m, n))], [np.zeros((n, m)), Ri]])
    At = np.block([[np.eye(m), A], [A.T, np.zeros((n, n))]])
    return ML @ At @ MR


def test_fgmres_is_exact_in_dimension_steps():
    P = randsvd_problem(8, 3, 1e2, seed=4)
    R, _ = _precond(P, 6)
    r = np.random.default_rng(0)
    f, h = r.standard_normal(8), r.standard_normal(3)
    dr, dx, info = fgmres.fgmres(P.A, R, f, h, 1e-14, 11)
    B = _dense_aug_prec(P.A, R)
    y = np.linalg.solve(B, np.concatenate([f, h]))
    assert np.allclose(dr, y[:8], atol=1e-10)
    assert np.allclose(dx, np.linalg.solve(R, y[8:]), atol=1e-10)


def test_fgmres_iterates_minimise_residual_over_krylov_space():
    P = randsvd_problem(20, 4, 1e2, seed=5)
    R, _ = _precond(P, 12)
    B = _dense_aug_prec(P.A, R)
    r = np.random.default_rng(1)
    rhs = r.standard_normal(24)
    prev = np.inf
    for k in (1, 3, 5, 8):
        dr, dx, info = fgmres.fgmres(P.A, R, rhs[:20], rhs[20:], 0.0, k)
        y = np.concatenate([dr, R @ dx])
        K = [rhs]
        for _ in range(k - 1):
            K.append(B @ K[-1])
        Kq = np.linalg.qr(np.column_stack(K))[0]
        c = np.linalg.lstsq(B @ Kq, rhs, rcond=None)[0]
        res_ref = np.linalg.norm(rhs - B @ (Kq @ c))
        res = np.linalg.norm(rhs - B @ y)
        assert abs(res - res_ref) <= 1e-10 * np.linalg.norm(rhs)
        assert abs(info["relres"] * np.linalg.norm(rhs) - res) <= 1e-10 * np.linalg.norm(rhs)
        assert res <= prev + 1e-14
        prev = res


def test_eq41_condition_number_of_preconditioned_augmented_matrix(golden):
    P = randsvd_problem(40, 5, 1e3, seed=6)
    R, _ = _precond(P, 20)
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    B = _dense_aug_prec(P.A, R)
    assert abs(np.linalg.cond(B) - theory.kappa_prec_aug(1.0, sv[0], sv[-1])) < 1e-8 * np.linalg.cond(B)
    assert np.linalg.cond(B) <= theory.kappa_prec_aug_bound(sv[0], 1 / sv[-1]) * (1 + 1e-12)
    # the paper's printed good-regime values are consistent with Eq. (4.1)
    v = {r[0]: float(r[1]) for r in golden("paper_fig3_good_regime.txt")}
    k = theory.kappa_prec_aug(1.0, v["norm_AR"], 1 / v["norm_AR_pinv"])
    assert abs(k - v["kappa_prec_aug"]) < 0.01 * v["kappa_prec_aug"]


def test_kappa_augmented_closed_form(golden):
    for kappa, printed in golden("paper_kappa_aug.txt"):
        assert abs(theory.kappa_aug(1.0, 1 / float(kappa)) - float(printed)) < 0.01 * float(printed)
    P = randsvd_problem(12, 4, 1e2, seed=7)
    At = np.block([[np.eye(12), P.A], [P.A.T, np.zeros((4, 4))]])
    assert abs(np.linalg.cond(At) - theory.kappa_aug(1.0, 1e-2)) < 1e-8 * np.linalg.cond(At)


def test_lsir_reaches_working_precision_in_one_step_paper_table3(golden):
    rows = [r for r in golden("paper_tables.txt") if r[0] in ("T3", "T4")]
    for table, kappa, us, u, _, lsir_its, gm_total in rows:
        kappa = float(kappa)
        fmt = {"half": "f16", "single": "f32", "double": "f64"}[us]
        dt = np.float32 if u == "single" else np.float64
        uu = 2.0 ** -24 if u == "single" else 2.0 ** -53
        tol = 1e-6 if u == "single" else 1e-12
        P = paper_problem(kappa, seed=0)
        xstar, rstar = exact.reference_solution(P.A, P.b)
        Y = sketch.sketch(P.A, P.b, 400, 0, fmt)
        R, c = qr.householder_qr(Y, 100, dtype=dt)
        # FGMRES's basis and rotations in FP64 (the GPU path's reading) and in u (the
        # paper's: everything but the three products in u, Sec. 4) give the printed counts
        for work in (np.float64, dt):
            x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), uu, tol, w_dtype=dt,
                                   us=rng.UNIT_ROUNDOFF[fmt], kappa=kappa, xstar=xstar, rstar=rstar,
                                   gm_work_dtype=work)
            assert info["converged"] and not info["escalated"]
            assert info["its"] == int(lsir_its), (table, kappa, info)
            assert abs(info["gmres_total"] - int(gm_total)) <= 3, (table, kappa, info)
            ex, er = exact.forward_errors(x, r, xstar, rstar)
            assert ex <= 4 * uu and er <= 4 * uu


def test_lsir_fails_where_paper_prints_dash():
    """Table 3: u_s half, u single, kappa >= 1e5 -> LSIR does not converge in 30 steps."""
    P = paper_problem(1e6, seed=0)
    xstar, rstar = exact.reference_solution(P.A, P.b)
    Y = sketch.sketch(P.A, P.b, 400, 0, "f16")
    R, c = qr.householder_qr(Y, 100, dtype=np.float32)
    x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -24, 1e-6,
                           w_dtype=np.float32, us=2.0 ** -11, kappa=1e6, xstar=xstar, rstar=rstar)
    assert not info["converged"] and not info["escalated"] and info["its"] == 30


def test_lsir_computable_stop_rule_reaches_target():
    P = randsvd_problem(600, 20, 1e4, rho=1e-3, seed=8)
    xstar, rstar = exact.reference_solution(P.A, P.b)
    R, xs = _precond(P, 80, fmt="f32")
    x, r, info = lsir.lsir(P.A, P.b, R, xs, 2.0 ** -24, 1e-6, w_dtype=np.float32)
    assert info["converged"]
    ex, er = exact.forward_errors(x, r, xstar, rstar)
    assert ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24


def test_escalation_rule_of_sec5():
    """Sec. 5: a refinement that does not converge is re-run from (x0, r0) with the FGMRES
    products in FP64 when kappa < 1/u_s, and not otherwise.  A cap of one step of two
    FGMRES iterations forces the first run to fail; the re-run, with the same caps, then
    starts from the same point with more accurate products."""
    P = paper_problem(1e2, seed=0)
    Y = sketch.sketch(P.A, P.b, 400, 0, "f16")
    R, c = qr.householder_qr(Y, 100, dtype=np.float32)
    xs = qr.sketch_and_solve(R, c)
    kw = dict(w_dtype=np.float32, ir_maxit=1, gm_maxit=2, us=2.0 ** -11)
    _, _, low = lsir.lsir(P.A, P.b, R, xs, 2.0 ** -24, 1e-6, kappa=1e2, escalate=False, **kw)
    assert not low["converged"] and not low["escalated"]
    # kappa u_s < 1: re-run with FP64 products; its steps equal an FP64-product run from the start
    xe, re, esc = lsir.lsir(P.A, P.b, R, xs, 2.0 ** -24, 1e-6, kappa=1e2, **kw)
    assert esc["escalated"] and esc["its"] == 1
    x64, r64, ref = lsir.lsir(P.A, P.b, R, xs, 2.0 ** -24, 1e-6, kappa=1e2, escalate=False,
                              op_dtype=np.float64, **kw)
    assert np.array_equal(xe, x64) and np.array_equal(re, r64)
    # kappa u_s >= 1 (1/u_s = 2048): no re-run
    _, _, no = lsir.lsir(P.A, P.b, R, xs, 2.0 ** -24, 1e-6, kappa=4096.0, **kw)
    assert not no["escalated"] and not no["converged"]
