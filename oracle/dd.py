"""Oracle: products in a precision beyond double, for u_A = u_L = u_R = quad (Sec. 5).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 5 reruns the refinement with the FGMRES products (the matrix-vector products with
A and A^T and the triangular solves with R) in quadruple precision when u is double
and the loop has not converged.  The GPU carries those products in double-double
(a value hi + lo, about 2^-106 relative).  This module computes them at least that
accurately from exact primitives, so that the oracle's result is the correctly rounded
(or DD-accurate) value and any GPU error shows against it:

* every product a * b is split exactly into p + e (``exact.two_product``),
* every sum of such terms is taken exactly by ``math.fsum`` (Shewchuk), and rounded once
  to a double, or to a double-double hi + lo with hi = fl(sum) and lo = fl(sum - hi),
* a double-double divided by a double is q1 + q2 with q1 = fl(hi / d) and q2 the rounded
  quotient of the exact remainder (hi + lo - q1 d) / d.

A double-double is a pair of float64 arrays (hi, lo) with |lo| <= ulp(hi) / 2.
"""
import math

import numpy as np

from .exact import two_product


def _dd_of_terms(terms):
    """(hi, lo) of the exact sum of the float64 ``terms``: hi = fl(S), lo = fl(S - hi)."""
    terms = list(terms)
    hi = math.fsum(terms)
    lo = math.fsum(terms + [-hi])
    return hi, lo


def _dd_div(hi, lo, d):
    """(hi + lo) / d as a double-double (the remainder is formed exactly)."""
    q1 = hi / d
    p, e = two_product(q1, d)
    rem = math.fsum([hi, lo, -float(p), -float(e)])
    q2 = rem / d
    s = q1 + q2
    return s, q2 - (s - q1)


def matvec(A, z_hi, z_lo=None, add=None, alpha=1.0):
    """Double-double w = alpha add + A (z_hi + z_lo), each row rounded once to (hi, lo).

    ``add`` (length m) enters the exact sum as the split product alpha * add."""
    A = np.asarray(A, np.float64)
    m, n = A.shape
    z_lo = np.zeros(n) if z_lo is None else np.asarray(z_lo, np.float64)
    p1, e1 = two_product(A, np.asarray(z_hi, np.float64)[None, :])
    p2, e2 = two_product(A, z_lo[None, :])
    if add is not None:
        pa, ea = two_product(np.float64(alpha), np.asarray(add, np.float64))
    hi = np.empty(m)
    lo = np.empty(m)
    for i in range(m):
        t = [p1[i], e1[i], p2[i], e2[i]]
        if add is not None:
            t.append([pa[i], ea[i]])
        hi[i], lo[i] = _dd_of_terms(np.concatenate(t).tolist())
    return hi, lo


def matvec_t(A, v):
    """Double-double A^T v (v a float64 vector), each entry rounded once."""
    A = np.asarray(A, np.float64)
    m, n = A.shape
    p, e = two_product(A, np.asarray(v, np.float64)[:, None])
    hi = np.empty(n)
    lo = np.empty(n)
    for j in range(n):
        hi[j], lo[j] = _dd_of_terms(np.concatenate([p[:, j], e[:, j]]).tolist())
    return hi, lo


def solve_upper(R, y_hi, y_lo=None):
    """Double-double x = R^-1 y, R upper triangular (float64): back substitution with
    each right-hand side y_i - sum_{k > i} R_ik x_k summed exactly, then divided."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    y_lo = np.zeros(n) if y_lo is None else np.asarray(y_lo, np.float64)
    xh = np.zeros(n)
    xl = np.zeros(n)
    for i in range(n - 1, -1, -1):
        row = R[i, i + 1:]
        p1, e1 = two_product(-row, xh[i + 1:])
        p2, e2 = two_product(-row, xl[i + 1:])
        h, l = _dd_of_terms([float(y_hi[i]), float(y_lo[i])] + p1.tolist() + e1.tolist()
                            + p2.tolist() + e2.tolist())
        xh[i], xl[i] = _dd_div(h, l, R[i, i])
    return xh, xl


def solve_upper_t(R, y_hi, y_lo=None):
    """Double-double x = R^-T y (forward substitution with the columns of R)."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    y_lo = np.zeros(n) if y_lo is None else np.asarray(y_lo, np.float64)
    xh = np.zeros(n)
    xl = np.zeros(n)
    for i in range(n):
        col = R[:i, i]
        p1, e1 = two_product(-col, xh[:i])
        p2, e2 = two_product(-col, xl[:i])
        h, l = _dd_of_terms([float(y_hi[i]), float(y_lo[i])] + p1.tolist() + e1.tolist()
                            + p2.tolist() + e2.tolist())
        xh[i], xl[i] = _dd_div(h, l, R[i, i])
    return xh, xl
