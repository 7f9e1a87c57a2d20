"""Pins for the oracle's extra-precise residuals and reference solution."""
from fractions import Fraction

import numpy as np
import pytest

from lsq_synth import randsvd_problem
from oracle import exact


def test_two_product_is_exact():
    r = np.random.default_rng(0)
    a = r.standard_normal(200) * 10 ** r.uniform(-5, 5, 200)
    b = r.standard_normal(200) * 10 ** r.uniform(-5, 5, 200)
    p, e = exact.two_product(a, b)
    for ai, bi, pi, ei in zip(a, b, p, e):
        assert Fraction(pi) + Fraction(ei) == Fraction(ai) * Fraction(bi)


def test_residual_aug_is_correctly_rounded():
    r = np.random.default_rng(1)
    A = r.standard_normal((9, 4))
    b, rr, x = r.standard_normal(9), r.standard_normal(9) * 1e-3, r.standard_normal(4)
    f, g = exact.residual_aug(A, b, rr, x)
    for i in range(9):
        ex = Fraction(b[i]) - Fraction(rr[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(4))
        assert f[i] == float(ex)
    for j in range(4):
        ex = -sum(Fraction(A[i, j]) * Fraction(rr[i]) for i in range(9))
        assert g[j] == float(ex)


def test_reference_solution_against_extended_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 300
    for kappa in (1e2, 1e8):
        P = randsvd_problem(25, 6, kappa, rho=1e-1, seed=2)
        x, r = exact.reference_solution(P.A, P.b)
        A = mp.matrix(P.A.tolist())
        b = mp.matrix(P.b.tolist())
        xe = mp.lu_solve(A.T * A, A.T * b)
        re = b - A * xe
        xe = np.array([float(v) for v in xe])
        re = np.array([float(v) for v in re])
        assert np.linalg.norm(x - xe) / np.linalg.norm(xe) < 4 * 2.0 ** -53
        assert np.linalg.norm(r - re) / np.linalg.norm(re) < 4 * 2.0 ** -53
