"""Oracle: extra-precise residuals and the reference solution x*, r*.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 5 measures every error against a 'true' solution from a 64-digit
solve.  This oracle plays that role for the stored FP64 data (A, b):

* ``residual_aug`` forms f = b - r - A x and g = -A^T r with every product
  split exactly into two doubles (Dekker's TwoProduct with Veltkamp's
  splitting) and every sum taken by ``math.fsum`` (Shewchuk's exactly
  rounded summation), so each entry is the correctly rounded value of the
  exact expression.  This is the residual in precision u_r of Alg. 2 (refinement residual)
  with u_r below double.
* ``reference_solution`` solves the LS problem by Householder QR of A
  (LAPACK through numpy, FP64) and refines it on the augmented system with
  those residuals (Bjorck, BIT 7, 1967), stopping when the correction is
  below 1e-17 relative.
"""
import math

import numpy as np

_SPLIT = 134217729.0   # 2^27 + 1 (Veltkamp splitting constant for binary64)


def two_product(a, b):
    """Exact a*b = p + e (Dekker), elementwise, without fused multiply-add."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    p = a * b
    ca = _SPLIT * a
    ah = ca - (ca - a)
    al = a - ah
    cb = _SPLIT * b
    bh = cb - (cb - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def residual_aug(A, b, r, x):
    """Correctly rounded f = b - r - A x and g = -A^T r (FP64 outputs)."""
    A = np.asarray(A, np.float64)
    m, n = A.shape
    b = np.asarray(b, np.float64)
    r = np.asarray(r, np.float64)
    x = np.asarray(x, np.float64)
    p, e = two_product(A, -x[None, :])            # rows: -A_i x split exactly
    f = np.empty(m)
    for i in range(m):
        f[i] = math.fsum(np.concatenate(([b[i], -r[i]], p[i], e[i])))
    pt, et = two_product(A, -r[:, None])          # columns: -A^T r split exactly
    g = np.empty(n)
    for j in range(n):
        g[j] = math.fsum(np.concatenate((pt[:, j], et[:, j])))
    return f, g


def residual(A, b, x):
    """Correctly rounded r = b - A x."""
    f, _ = residual_aug(A, b, np.zeros(len(b)), x)
    return f


def reference_solution(A, b, maxit=12):
    """x*, r* for the stored FP64 (A, b): QR solve + augmented refinement."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    Q, R = np.linalg.qr(A, mode="reduced")
    x = np.linalg.solve(R, Q.T @ b)
    r = residual(A, b, x)
    for _ in range(maxit):
        f, g = residual_aug(A, b, r, x)
        h = np.linalg.solve(R.T, g)              # R^-T g
        d = Q.T @ f
        dx = np.linalg.solve(R, d - h)
        dr = f - Q @ (d - h)
        x = x + dx
        r = r + dr
        if np.linalg.norm(dx) <= 1e-17 * np.linalg.norm(x) and \
           np.linalg.norm(dr) <= 1e-17 * max(np.linalg.norm(r), 1e-300):
            break
    return x, r


def forward_errors(x, r, xstar, rstar):
    """Relative forward errors ||x - x*||/||x*||, ||r - r*||/||r*|| (Sec. 5)."""
    ex = np.linalg.norm(np.asarray(x) - xstar) / np.linalg.norm(xstar)
    nr = np.linalg.norm(rstar)
    er = np.linalg.norm(np.asarray(r) - rstar) / nr if nr > 0 else 0.0
    return float(ex), float(er)
