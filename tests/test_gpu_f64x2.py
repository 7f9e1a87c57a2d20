"""u = double with double-double residuals and FGMRES products (Sec. 5, Table 4) and the
alpha-scaled augmented system (Sec. 4.1), through the C ABI against the oracle.

* lsq_residual in u_r = double-double against the correctly rounded residual
  (``exact.residual_aug``): within one rounding plus the double-double sum error
  (about 3 * 2^-106 of the terms per addition); u_r = double within the FP64
  dot-product bound.
* One refinement step with the alpha-scaled system and with double-double products
  against ``oracle.lsir.refine`` with the same alpha / with ``op_dtype="dd"``, compared
  in FGMRES's own variables [dr/alpha; R dx] like the FP64 step test.  With
  double-double products the residual correction dr is within 20 k kappa_p u (FP64
  products would leave kappa(A) u in A z); R dx keeps the kappa(R) u of storing
  z_j = R^-1 v_j in FP64.
* lsq_lsir with (u_s, u, u_r) = (double, double, quad) on the paper's problems reaches
  4u, and at kappa = 1e12 (a starred row of Table 4) it needs, and takes, the re-run
  with double-double products.
"""
import numpy as np
import pytest
import torch

from conftest import colmajor, dev
from lsq_synth import paper_problem, randsvd_problem
from oracle import exact, lsir, qr, sketch, theory

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("ur", ["f64x2", "f64"])
def test_residual_against_correctly_rounded(lsq, handle, ur):
    m, n = 3000, 70
    P = randsvd_problem(m, n, 1e8, rho=1e-6, seed=5)
    # near the least-squares solution the residual cancels: f and g are far below their terms
    x = np.linalg.lstsq(P.A, P.b, rcond=None)[0]
    r = P.b - P.A @ x
    x = x * (1 + 1e-14 * np.random.default_rng(0).standard_normal(n))
    f_ex, g_ex = exact.residual_aug(P.A, P.b, r, x)
    f, g = zeros(m), zeros(n)
    st = lsq.lsq_residual(handle, dev(P.A), dev(P.b), m, n, ur, None, dev(x), dev(r), f, g)
    assert st == 0
    f, g = f.cpu().numpy(), g.cpu().numpy()
    rows = np.abs(P.b) + np.abs(r) + np.abs(P.A) @ np.abs(x)
    cols = np.abs(P.A).T @ np.abs(r)
    assert np.max(np.abs(f_ex) / rows) < 1e-6      # the cancellation is real
    if ur == "f64x2":
        assert np.all(np.abs(f - f_ex) <= U64 * np.abs(f_ex) + (n + 3) * 2.0 ** -102 * rows)
        assert np.all(np.abs(g - g_ex) <= U64 * np.abs(g_ex) + (m + 1024) * 2.0 ** -102 * cols)
    else:
        assert np.all(np.abs(f - f_ex) <= (n + 3) * U64 * rows)
        assert np.all(np.abs(g - g_ex) <= (m + 1024) * U64 * cols)


def _setup(m, n, kappa, seed):
    P = randsvd_problem(m, n, kappa, rho=1e-3, seed=seed)
    s = 4 * n
    Y = sketch.sketch(P.A, P.b, s, 5, "f64")
    R, c = qr.householder_qr(Y, n)
    x0 = qr.sketch_and_solve(R, c)
    r0 = P.b - P.A @ x0
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    return P, s, R, x0, r0, sv


def _compare_step(x, r, x0, r0, xo, ro, R, alpha, bound):
    dxg, drg = x.cpu().numpy() - x0, r.cpu().numpy() - r0
    dg = np.concatenate([drg / alpha, R @ dxg])
    do = np.concatenate([(ro - r0) / alpha, R @ (xo - x0)])
    rel = np.linalg.norm(dg - do) / np.linalg.norm(do)
    assert rel <= bound, (rel, bound)
    return rel


@pytest.mark.parametrize("alpha", [0.25, 3.0])
def test_scaled_refinement_step_matches_oracle(lsq, handle, alpha):
    m, n, kappa = 3000, 60, 1e6
    P, s, R, x0, r0, sv = _setup(m, n, kappa, seed=11)
    tol = 1e-10
    xo, ro, io = lsir.refine(P.A, P.b, R, x0, r0, U64, tol, 1, 50, np.float64, "f64", alpha=alpha)
    x, r = dev(x0), dev(r0)
    st, info = lsq.lsq_ir_step(handle, dev(P.A), dev(P.b), m, n, s, "f64", "f64", "f64", "f64", tol, 5,
                               {"gmres_maxit": 50, "aug_alpha": alpha}, dev(colmajor(R)), x, r)
    kg, ko = info.gmres_its[0], io["gmres_its"][0]
    assert info.aug_alpha == alpha
    assert abs(kg - ko) <= 1, (kg, ko)
    kp = theory.kappa_prec_aug(alpha, sv[0], sv[-1])
    bound = 20 * (max(kg, ko) * kp + np.linalg.cond(R)) * U64 + (tol * kp if kg != ko else 0.0)
    rel = _compare_step(x, r, x0, r0, xo, ro, R, alpha, bound)
    print("alpha", alpha, "its", kg, "kappa_p", kp, "rel", rel, "bound", bound)


def test_double_double_products_step_matches_oracle(lsq, handle):
    """u_A = u_L = u_R = double-double (the Sec. 5 re-run for u = double) with
    u_r = double-double and h = R^-T g in u_r on both sides, against the oracle's
    exact-sum products."""
    m, n, kappa = 2000, 40, 1e10
    P, s, R, _, _, sv = _setup(m, n, kappa, seed=12)
    # from (x, r) = (0, 0) the update x + dx, r + dr is exact on both sides, so the
    # corrections themselves are compared (after a general start, the FP64 rounding of
    # x + dx alone is ||R|| u ||x|| in these variables)
    x0, r0 = np.zeros(n), np.zeros(m)
    tol = 1e-12
    xo, ro, io = lsir.refine(P.A, P.b, R, x0, r0, U64, tol, 1, 50, "dd", "exact", h_ur=True)
    x, r = dev(x0), dev(r0)
    st, info = lsq.lsq_ir_step(handle, dev(P.A), dev(P.b), m, n, s, "f64", "f64", "f64", "f64x2", tol, 5,
                               {"gmres_maxit": 50, "ops_escalated": 1, "h_in_ur": 1}, dev(colmajor(R)), x, r)
    kg, ko = info.gmres_its[0], io["gmres_its"][0]
    assert abs(kg - ko) <= 1, (kg, ko)
    kp = theory.kappa_prec_aug(1.0, sv[0], sv[-1])
    # dr = V_top y: the basis, Gram-Schmidt and rotations (FP64 on both sides) and the
    # products A z, which double-double makes exact to working precision; FP64 products
    # would leave kappa(A) u = 1e-6 of |A||z| in w_top (|A z| ~ |v|, |A||z| ~ kappa |v|):
    # the oracle's own FP64-product step lands 1.7e-5 from its double-double one here
    bound = 20 * max(kg, ko) * kp * U64 + (tol * kp if kg != ko else 0.0)
    assert kappa * U64 > 100 * bound
    dr_g, dr_o = r.cpu().numpy(), ro
    rel_r = np.linalg.norm(dr_g - dr_o) / np.linalg.norm(dr_o)
    assert rel_r <= bound, (rel_r, bound)
    # R dx = R Z y: Z holds z_j = R^-1 v_j rounded to FP64 (the working precision of the
    # basis, as in the oracle), which leaves ||R|| u ||z_j|| per column: kappa(R) u
    rel = _compare_step(x, r, x0, r0, xo, ro, R, 1.0, 20 * (max(kg, ko) * kp + np.linalg.cond(R)) * U64)
    print("dd its", kg, ko, "kappa_p", kp, "rel_r", rel_r, "bound", bound, "rel", rel)


@pytest.mark.parametrize("kappa", [1e2, 1e10])
def test_lsir_u_double_reaches_4u(lsq, handle, kappa):
    """Table 4 setting (u_s = u = double, u_r = quad): forward errors <= 4u without the re-run."""
    P = paper_problem(kappa, seed=0)
    m, n = P.A.shape
    xstar, rstar = exact.reference_solution(P.A, P.b)
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, 4 * n, "f64", "f64", "f64", "f64x2", 1e-12, 0,
                            None, x, r)
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
    print(kappa, info.as_dict()["gmres_its"], info.escalated, ex, er)
    assert st == 0 and info.ir_converged == 1 and info.escalated == 0
    assert ex <= 4 * U64 and er <= 4 * U64, (ex, er)


def test_lsir_u_double_starred_row_escalates_to_double_double(lsq, handle):
    """Table 4 at kappa = 1e12 (2*, 138*): the FP64-product refinement does not reach the
    stopping rule in 30 steps; the re-run with double-double products (<= 80 FGMRES
    iterations per step) converges to 4u."""
    P = paper_problem(1e12, seed=0)
    m, n = P.A.shape
    xstar, rstar = exact.reference_solution(P.A, P.b)
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, 4 * n, "f64", "f64", "f64", "f64x2", 1e-12, 0,
                            None, x, r)
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
    d = info.as_dict()
    print(d["gmres_its"], info.escalated, ex, er)
    assert st == 0 and info.escalated == 1 and info.ir_converged == 1
    assert all(k <= 80 for k in d["gmres_its"]) and info.ir_its <= 4
    assert ex <= 4 * U64 and er <= 4 * U64, (ex, er)
