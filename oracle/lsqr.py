"""Oracle: Algorithm 2 (the LSQR start) -- LSQR right-preconditioned by R.

Test infrastructure only (see ``oracle/__init__.py``).

LSQR of Paige & Saunders (ACM TOMS 8, 1982) applied to the preconditioned
operator Ahat = A R^-1, started from x0 (the sketch-and-solve x_s of Sec. 4):
it solves min_z || (b - A x0) - Ahat z || and returns x = x0 + R^-1 z.

Stopping (the paper runs MATLAB's lsqr for at most 2n iterations with tol
1e-6 for single and 1e-12 for double working precision, Sec. 5; MATLAB's
tests are the two Paige-Saunders tests).  The reading taken here:
  S1: ||r_k|| <= tol ||b||,
  S2: ||Ahat^T r_k|| <= tol * ||Ahat||_est * ||r_k||,
where r_k = b - A x_k (= phibar), ||Ahat^T r_k|| = phibar * alpha * |c|, and
||Ahat||_est = sqrt(sum of alpha_i^2 + beta_i^2) (the Frobenius-type estimate
the bidiagonalisation provides).
"""
import numpy as np

from .qr import solve_upper, solve_upper_t


def lsqr(A, b, R, x0, tol, maxit, dtype=np.float64):
    """Preconditioned LSQR.  Returns (x, info) with x in FP64.

    ``dtype`` is the working precision u (float64 or float32): A, R, b and
    all vectors are held in it (Sec. 5 stores A and b in single when u is
    single).  info = dict(its, flag, normr, normar, normA).
    """
    Aw = np.asarray(A, dtype=dtype)
    Rw = np.asarray(R, dtype=dtype)
    bw = np.asarray(b, dtype=dtype)
    x0w = np.asarray(x0, dtype=dtype)

    def prec(v):       # R^-1 v in precision dtype
        return solve_upper(Rw, v).astype(dtype)

    def prec_t(v):     # R^-T v
        return solve_upper_t(Rw, v).astype(dtype)

    normb = float(np.linalg.norm(bw.astype(np.float64)))
    rbar = bw - Aw @ x0w
    beta = dtype(np.linalg.norm(rbar))
    u = rbar / beta if beta > 0 else rbar
    v = prec_t(Aw.T @ u)
    alpha = dtype(np.linalg.norm(v))
    if alpha > 0:
        v = v / alpha
    w = v.copy()
    z = np.zeros(Aw.shape[1], dtype=dtype)
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    info = dict(its=0, flag=0, normr=float(beta), normar=float(alpha * beta), normA=0.0)
    if beta == 0 or alpha == 0:
        info["flag"] = 1
        return x0w.astype(np.float64), info
    for k in range(1, maxit + 1):
        # bidiagonalisation: beta u = Ahat v - alpha u ; alpha v = Ahat^T u - beta v
        uu = Aw @ prec(v) - alpha * u
        beta = dtype(np.linalg.norm(uu))
        if beta > 0:
            u = uu / beta
        anorm2 += float(alpha) ** 2 + float(beta) ** 2
        vv = prec_t(Aw.T @ u) - beta * v
        alpha = dtype(np.linalg.norm(vv))
        if alpha > 0:
            v = vv / alpha
        # plane rotation eliminating beta
        rho = dtype(np.sqrt(rhobar * rhobar + beta * beta))
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        z = z + (phi / rho) * w
        w = v - (theta / rho) * w
        normr = float(abs(phibar))
        normar = float(abs(phibar * alpha * c))
        normA = np.sqrt(anorm2)
        info.update(its=k, normr=normr, normar=normar, normA=normA)
        if normr <= tol * normb:
            info["flag"] = 1
            break
        if normar <= tol * normA * normr:
            info["flag"] = 2
            break
        if beta == 0 or alpha == 0:
            info["flag"] = 3
            break
    x = x0w.astype(np.float64) + solve_upper(np.asarray(R, np.float64), z.astype(np.float64))
    return x, info
