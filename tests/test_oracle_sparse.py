"""Pins of the oracle's sparse sign embedding (Sec. 2) against what the definition and the
mathematics fix: structure of Omega, uniform and independent choices, the isometry in
expectation, the exact fixed-point rounding, the overflow margin, Sec. 2's identity
kappa(A R^-1) = kappa(Omega U), and the embedding quality of a zeta = 8 sketch."""
from fractions import Fraction

import numpy as np
import pytest

from lsq_synth import randsvd_problem
from oracle import qr, sparse, theory


def test_each_column_has_zeta_distinct_signed_entries():
    for s, zeta in ((40, 8), (9, 8), (8, 8), (5, 2), (3, 1)):
        Om = sparse.dense_omega(500, s, zeta, seed=3)
        nz = Om != 0
        assert np.all(nz.sum(axis=0) == zeta)                    # zeta rows, all distinct
        assert np.allclose(np.abs(Om[nz]), 1 / np.sqrt(zeta))    # +-zeta^-1/2
        assert np.allclose(np.linalg.norm(Om, axis=0), 1.0)      # unit columns: E||Omega x||^2 = ||x||^2


def test_choices_are_uniform_and_signs_balanced():
    m, s, zeta = 200_000, 64, 8
    rows, signs = sparse.sparse_rows(m, s, zeta, seed=11)
    counts = sparse.row_counts(rows, s)
    exp = m * zeta / s
    chi2 = np.sum((counts - exp) ** 2 / exp)
    assert chi2 < s - 1 + 6 * np.sqrt(2 * (s - 1))               # chi-square, s - 1 d.o.f., ~6 sigma
    frac_neg = np.mean(signs < 0)
    assert abs(frac_neg - 0.5) < 6 * np.sqrt(0.25 / signs.size)
    # Floyd's algorithm draws a uniform subset (not uniform slots): with s = 5, zeta = 2
    # each of the 10 subsets is equally likely
    r5, _ = sparse.sparse_rows(100_000, 5, 2, seed=13)
    key = np.minimum(r5[:, 0], r5[:, 1]) * 5 + np.maximum(r5[:, 0], r5[:, 1])
    cnt = np.array([np.sum(key == a * 5 + b) for a in range(5) for b in range(a + 1, 5)])
    assert cnt.sum() == 100_000 and np.sum((cnt - 1e4) ** 2 / 1e4) < 9 + 6 * np.sqrt(18)
    # different seeds, different matrices; same seed, same matrix
    r2, _ = sparse.sparse_rows(m, s, zeta, seed=12)
    r1, _ = sparse.sparse_rows(m, s, zeta, seed=11)
    assert np.array_equal(r1, rows) and not np.array_equal(r2, rows)


def test_isometry_in_expectation():
    r = np.random.default_rng(0)
    x = r.standard_normal(3000)
    vals = [np.linalg.norm(sparse.dense_omega(3000, 60, 8, seed=sd) @ x) ** 2 for sd in range(40)]
    nx = np.linalg.norm(x) ** 2
    # E ||Omega x||^2 = ||x||^2 exactly (unit columns, independent signs); the sample mean
    # of 40 draws is within 4 standard errors
    assert abs(np.mean(vals) - nx) < 4 * np.std(vals) / np.sqrt(len(vals))


def test_grid_rounding_is_exact_round_half_even():
    r = np.random.default_rng(5)
    x = np.concatenate([r.standard_normal(3000) * np.exp(r.uniform(-30, 30, 3000)),
                        [0.0, -0.0, 0.5, 1.5, 2.5, -0.5, -1.5, 5e-324, -5e-324, 2.0 ** -1074 * 3]])
    for q in (0, 10, 40, -20, 1070, 1100):
        got = sparse.to_grid(x, q)
        for xv, g in zip(x[:400].tolist() + x[-10:].tolist(), got[:400].tolist() + got[-10:].tolist()):
            v = Fraction(xv) * Fraction(2) ** q
            if abs(v) >= 2 ** 62:
                continue
            fl = v.numerator // v.denominator
            rem = v - fl
            want = fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1) else 0)
            assert g == want, (xv, q, g, want)


def test_grid_leaves_room_for_every_partial_sum():
    P = randsvd_problem(5000, 30, 1e4, seed=2)
    rows, _ = sparse.sparse_rows(5000, 120, 8, seed=1)
    mc = sparse.row_counts(rows, 120).max()
    Ab = np.column_stack([P.A, P.b])
    q = sparse.grid_exponents(Ab, mc)
    Q = np.stack([sparse.to_grid(Ab[:, c], q[c]) for c in range(31)], axis=1)
    assert np.abs(Q).max() * mc < 2 ** 62
    # and the grid is fine: every column is represented to 2^-(61 - h) of its largest entry
    h = int(mc).bit_length()
    assert np.all(np.abs(np.ldexp(Q.astype(np.float64), -q[None, :]) - Ab)
                  <= np.ldexp(1.0, -(61 - h)) * np.abs(Ab).max(axis=0)[None, :])


def test_sketch_equals_the_dense_product():
    P = randsvd_problem(4000, 20, 1e3, rho=1e-2, seed=4)
    s, zeta = 80, 8
    Y = sparse.sparse_sketch(P.A, P.b, s, zeta, seed=9)
    Om = sparse.dense_omega(4000, s, zeta, seed=9)
    Yd = Om @ np.column_stack([P.A, P.b])
    # the only differences: the grid (2^-(61-h) of each column's largest entry, per entry)
    # and the final rounding
    mag = np.abs(Om) @ np.abs(np.column_stack([P.A, P.b]))
    assert np.all(np.abs(Y - Yd) <= 2.0 ** -45 * mag + 1e-300)


def test_kappa_identity_and_embedding_quality():
    """Sec. 2: kappa(A R^-1) = kappa(Omega U) for the R of Omega A; a zeta = 8 sparse sign
    sketch with s = 4n stays near the Gaussian (Marchenko-Pastur) value."""
    m, n, s = 20000, 50, 200
    P = randsvd_problem(m, n, 1e10, rho=1e-3, seed=6)
    Y = sparse.sparse_sketch(P.A, P.b, s, 8, seed=2)
    R, _ = qr.householder_qr(Y, n)
    sv = np.linalg.svd(np.linalg.solve(R.T, P.A.T).T, compute_uv=False)
    kar = sv[0] / sv[-1]
    U, _, _ = np.linalg.svd(P.A, full_matrices=False)
    Om = sparse.dense_omega(m, s, 8, seed=2)
    su = np.linalg.svd(Om @ U, compute_uv=False)
    assert kar == pytest.approx(su[0] / su[-1], rel=1e-3)
    assert kar <= 1.3 * theory.mp_limits(n, s)[2]


def test_split_halves_sum_equals_plain_integer_sum():
    """The oracle's exact sums (FP64 bincount of 31-bit halves) equal plain int64 scatter-adds."""
    from lsq_synth import randsvd_problem as rp
    P = rp(3000, 12, 1e3, seed=1)
    Y = sparse.sparse_sketch(P.A, P.b, 60, 8, 5)
    Ab = np.column_stack([P.A, P.b])
    rows, signs = sparse.sparse_rows(3000, 60, 8, 5)
    q = sparse.grid_exponents(Ab, sparse.row_counts(rows, 60).max())
    Q = np.stack([sparse.to_grid(Ab[:, c], q[c]) for c in range(13)], axis=1)
    acc = np.zeros((60, 13), dtype=np.int64)
    for k in range(8):
        np.add.at(acc, rows[:, k], signs[:, k:k + 1] * Q)
    assert np.array_equal(Y, np.ldexp(acc.astype(np.float64), -q[None, :]) * (1.0 / np.sqrt(8.0)))
