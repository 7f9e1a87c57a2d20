"""Oracle: Algorithm 1 (the QR of the sketch) -- Householder QR of the sketch, R only.

Test infrastructure only (see ``oracle/__init__.py``).

Alg. 1 asks for the R factor of an economic Householder QR of Y = Omega A in
precision u_QR (the proof of Thm. 3.1 uses the Householder error analysis of
Higham, Thm. 19.4).  Sec. 4 starts LSQR from the sketch-and-solve solution
x_s = R^-1 (Q^T Omega b): the same reflectors are applied to the sketched
right-hand side (column n of Y), so Q itself is never formed.

Reflector for column k (Golub & Van Loan): x = Y[k:, k],
v = x + sign(x_1) ||x|| e_1 with sign(0) = +1, H = I - 2 v v^T / v^T v, so
H x = -sign(x_1) ||x|| e_1.  R is unique only up to the signs of its rows;
the result is normalised to a non-negative diagonal (row k of R and entry k
of c flip together, which leaves R^-1 c unchanged).
"""
import numpy as np


def householder_qr(Y, n, dtype=np.float64):
    """Return (R, c): R (n x n, upper, diag >= 0) and c = (Q^T Y[:, n])[:n].

    Y has n + 1 columns (the last one is Omega b) or n columns (c = None).
    ``dtype`` is the arithmetic precision u_QR (float64 or float32).
    """
    W = np.array(Y, dtype=dtype, copy=True)
    s = W.shape[0]
    for k in range(n):
        x = W[k:, k].copy()
        alpha = np.sqrt(np.dot(x, x))
        sgn = dtype(1.0) if x[0] >= 0 else dtype(-1.0)
        v = x
        v[0] = x[0] + sgn * alpha
        vtv = np.dot(v, v)
        if vtv == 0:
            continue
        # apply H = I - 2 v v^T / (v^T v) to the trailing columns (incl. rhs)
        T = W[k:, k:]
        wT = (v @ T) * (dtype(2.0) / vtv)
        T -= np.outer(v, wT)
        W[k + 1:, k] = 0
    R = np.triu(W[:n, :n]).astype(np.float64)
    c = W[:n, n].astype(np.float64) if W.shape[1] > n else None
    sign = np.where(np.diag(R) < 0, -1.0, 1.0)
    R = R * sign[:, None]
    if c is not None:
        c = c * sign
    return R, c


def solve_upper(R, y):
    """x = R^-1 y by back substitution (FP64)."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    x = np.array(y, dtype=np.float64, copy=True)
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - np.dot(R[i, i + 1:], x[i + 1:])) / R[i, i]
    return x


def solve_upper_t(R, y):
    """x = R^-T y by forward substitution (FP64)."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    x = np.array(y, dtype=np.float64, copy=True)
    for i in range(n):
        x[i] = (x[i] - np.dot(R[:i, i], x[:i])) / R[i, i]
    return x


def sketch_and_solve(R, c):
    """x_s = R^-1 c (Sec. 4, the LSQR starting vector of Alg. 2)."""
    return solve_upper(R, c)
