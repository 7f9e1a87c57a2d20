"""Pins of the oracle's double-double products (Sec. 5: u_A = u_L = u_R = quad for u double)
and of the alpha-scaled augmented system (Sec. 4.1), against exact rational arithmetic,
the eigenvalues of the scaled matrix, and Table 4's starred rows."""
from fractions import Fraction

import numpy as np

from lsq_synth import paper_problem, randsvd_problem
from oracle import dd, exact, fgmres, lsir, qr, sketch, theory


def test_dd_matvec_is_the_correctly_rounded_exact_sum():
    r = np.random.default_rng(1)
    m, n = 25, 9
    A = r.standard_normal((m, n)) * np.exp(r.uniform(-20, 20, (m, n)))
    zh = r.standard_normal(n)
    zl = zh * 2.0 ** -60 * r.standard_normal(n)
    add = r.standard_normal(m)
    alpha = 0.375
    # a row with near-total cancellation: its value is far below the terms
    A[3, 0] = -(alpha * add[3] + np.dot(A[3, 1:], zh[1:])) / zh[0]
    hi, lo = dd.matvec(A, zh, zl, add=add, alpha=alpha)
    for i in range(m):
        ex = Fraction(alpha) * Fraction(float(add[i])) + sum(
            Fraction(float(A[i, j])) * (Fraction(float(zh[j])) + Fraction(float(zl[j]))) for j in range(n))
        assert hi[i] == float(ex), i                       # float(Fraction) rounds to nearest
        assert lo[i] == float(ex - Fraction(float(hi[i]))), i
    th, tl = dd.matvec_t(A, add)
    for j in range(n):
        ex = sum(Fraction(float(A[i, j])) * Fraction(float(add[i])) for i in range(m))
        assert th[j] == float(ex) and tl[j] == float(ex - Fraction(float(th[j])))


def test_dd_triangular_solves_against_exact_rationals():
    r = np.random.default_rng(2)
    n = 7
    for cond_scale in (1.0, 1e6):
        R = np.triu(r.standard_normal((n, n)))
        R[np.diag_indices(n)] = np.abs(R[np.diag_indices(n)]) + 1.0
        R[-1, -1] /= cond_scale
        yh = r.standard_normal(n)
        yl = yh * 2.0 ** -55 * r.uniform(-1, 1, n)
        kR = np.linalg.cond(R)
        for solve, upper in ((dd.solve_upper, True), (dd.solve_upper_t, False)):
            xh, xl = solve(R, yh, yl)
            Rf = [[Fraction(float(R[i, j])) for j in range(n)] for i in range(n)]
            y = [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(yh, yl)]
            x = [Fraction(0)] * n
            order = range(n - 1, -1, -1) if upper else range(n)
            for i in order:
                ks = range(i + 1, n) if upper else range(i)
                s = y[i] - sum((Rf[i][k] if upper else Rf[k][i]) * x[k] for k in ks)
                x[i] = s / Rf[i][i]
            xmax = max(abs(v) for v in x)
            err = max(abs(Fraction(float(a)) + Fraction(float(b)) - v) for a, b, v in zip(xh, xl, x))
            # double-double: about 2^-104 per operation, amplified by kappa(R) at most
            assert err <= Fraction(2) ** -100 * Fraction(float(kR)) * xmax, (upper, cond_scale, float(err / xmax))
            assert all(abs(b) <= abs(a) * 2.0 ** -52 for a, b in zip(xh, xl))


def test_scaled_augmented_condition_number_sec41():
    """kappa of [[alpha I, A R^-1], [R^-T A^T, 0]] equals the closed form for every alpha
    (denominator min(2 alpha, ...): the eigenvalues are alpha and (alpha +- sqrt(alpha^2 +
    4 sigma_i^2)) / 2), and the optimal alpha = sigma_min / sqrt(2) gives at most
    2 kappa(A R^-1)."""
    P = randsvd_problem(60, 6, 1e4, seed=3)
    Y = sketch.sketch(P.A, P.b, 24, 1, "f16")          # a rough R: kappa(A R^-1) well above 1
    R, _ = qr.householder_qr(Y, 6)
    B = P.A @ np.linalg.inv(R)
    sv = np.linalg.svd(B, compute_uv=False)
    for alpha in (0.05, 0.3, 1.0, 2.5, sv[-1] / np.sqrt(2)):
        M = np.block([[alpha * np.eye(60), B], [B.T, np.zeros((6, 6))]])
        k = np.linalg.cond(M)
        assert abs(k - theory.kappa_prec_aug(alpha, sv[0], sv[-1])) <= 1e-8 * k, alpha
    k_opt = theory.kappa_prec_aug(sv[-1] / np.sqrt(2), sv[0], sv[-1])
    assert k_opt <= 2 * sv[0] / sv[-1] * (1 + 1e-12)
    assert theory.kappa_prec_aug(1.0, sv[0], sv[-1]) > k_opt


def test_scaled_fgmres_gives_the_unscaled_correction():
    """FGMRES on the alpha-scaled system returns the same (dr, dx) (exact in m + n steps)."""
    P = randsvd_problem(9, 3, 1e2, seed=4)
    Y = sketch.sketch(P.A, P.b, 6, 0, "f64")
    R, _ = qr.householder_qr(Y, 3)
    r = np.random.default_rng(0)
    f, h = r.standard_normal(9), r.standard_normal(3)
    At = np.block([[np.eye(9), P.A], [P.A.T, np.zeros((3, 3))]])
    d = np.linalg.solve(At, np.concatenate([f, R.T @ h]))     # [dr; dx] of the unscaled system
    for alpha in (0.2, 1.0, 3.0):
        dr, dx, info = fgmres.fgmres(P.A, R, f, h, 1e-15, 12, alpha=alpha)
        assert np.allclose(dr, d[:9], atol=1e-10) and np.allclose(dx, d[9:], atol=1e-10), alpha


def test_quad_products_reproduce_table4_starred_rows(golden):
    """Table 4, u_s = u = double, kappa >= 1e12: LSIR does not converge with FP64
    products; with u_A = u_L = u_R = quad (double-double here) and at most 80 FGMRES
    iterations it converges in the printed number of refinement steps, with the
    printed FGMRES total within 5."""
    rows = [r for r in golden("paper_tables.txt") if r[0] == "T4*"]
    assert rows
    for _, kappa, us, u, _, lsir_its, gm_total in rows:
        kappa = float(kappa)
        P = paper_problem(kappa, seed=0)
        xstar, rstar = exact.reference_solution(P.A, P.b)
        Y = sketch.sketch(P.A, P.b, 400, 0, "f64")
        R, c = qr.householder_qr(Y, 100)
        x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -53, 1e-12,
                               w_dtype=np.float64, us=2.0 ** -53, kappa=kappa, xstar=xstar, rstar=rstar)
        assert info["escalated"] and info["converged"], (kappa, info)
        assert info["its"] == int(lsir_its), (kappa, info)
        assert abs(info["gmres_total"] - int(gm_total)) <= 5, (kappa, info)
        ex, er = exact.forward_errors(x, r, xstar, rstar)
        assert ex <= 4 * 2.0 ** -53 and er <= 4 * 2.0 ** -53


def test_h_in_quad_reading_converges_at_least_as_fast():
    """Alg. 2 marks h = R^-T g with u_r; solved that way (double-double from the
    double-double g) the escalated refinement at kappa = 1e12 needs fewer steps than the
    printed 2* (the FP64 solve of the default reading reproduces the printed count)."""
    kappa = 1e12
    P = paper_problem(kappa, seed=0)
    xstar, rstar = exact.reference_solution(P.A, P.b)
    Y = sketch.sketch(P.A, P.b, 400, 0, "f64")
    R, c = qr.householder_qr(Y, 100)
    x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -53, 1e-12, w_dtype=np.float64,
                           us=2.0 ** -53, kappa=kappa, xstar=xstar, rstar=rstar, h_ur=True)
    assert info["escalated"] and info["converged"] and info["its"] <= 2
    ex, er = exact.forward_errors(x, r, xstar, rstar)
    assert ex <= 4 * 2.0 ** -53 and er <= 4 * 2.0 ** -53
