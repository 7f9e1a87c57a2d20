"""Oracle: Algorithm 2 (the FGMRES solve) -- split-preconditioned FGMRES on the augmented system.

Test infrastructure only (see ``oracle/__init__.py``).

Eq. (1.2) defines the preconditioned augmented system
    M_L^-1 Atilde M_R^-1 y = s,   Atilde = [[I, A], [A^T, 0]],
    M_L^-1 = diag(I, R^-T),   M_R^-1 = diag(I, R^-1),
solved by flexible GMRES (Saad, SIAM J. Sci. Comput. 14, 1993) because the
right preconditioner is applied inexactly (precision u_R).  FGMRES keeps the
preconditioned vectors z_j = M_R^-1 v_j and returns the correction
d = Z_k y_k = [delta r; delta x] directly; the top block of z_j equals that of
v_j, so only the bottom n x k block of Z is kept.

Readings where the paper is silent: x0 = 0, no restart, modified
Gram-Schmidt Arnoldi and Givens rotations in FP64, stop when the residual
estimate |g_{k+1}| <= tol ||s||, at most ``maxit`` iterations (50 in Sec. 5).
The products with Atilde, M_L^-1 and M_R^-1 are formed in ``op_dtype``
(u_A = u_L = u_R).  ``work_dtype`` is the precision of everything else (the
basis, the Gram-Schmidt and the rotations): FP64 by default (the GPU path's
choice); the paper's own setting (Sec. 4: the remaining computations in u) is
``work_dtype = u``.

Scaling (Sec. 4.1): with ``alpha`` != 1 the system solved is the scaled one,
M_L^-1 Atilde_alpha M_R^-1 [dr / alpha; dz] = [f; h / alpha] with
Atilde_alpha = [[alpha I, A], [A^T, 0]]: the same correction, since alpha (dr / alpha)
+ A dx = f and A^T (dr / alpha) = g / alpha.  Sec. 5 runs alpha = 1.

``op_dtype = "dd"`` takes the three products in double-double or better
(``oracle.dd``: exact splits and sums), each rounded once to FP64 where FGMRES stores
it: Sec. 5's escalated setting u_A = u_L = u_R = quad for u = double.
"""
import numpy as np

from . import dd
from .qr import solve_upper, solve_upper_t


def fgmres(A, R, f, h, tol, maxit, op_dtype=np.float64, work_dtype=np.float64, alpha=1.0):
    """Solve M_L^-1 Atilde_alpha M_R^-1 y = [f; h / alpha]; return (dr, dx, info) with
    dr = alpha y_top (alpha = 1: the unscaled system of Eq. (1.2))."""
    wd = work_dtype
    A64 = np.asarray(A, dtype=np.float64)
    m, n = A64.shape
    quad = isinstance(op_dtype, str) and op_dtype == "dd"
    Ao = A64 if quad else A64.astype(op_dtype)
    Ro = np.asarray(R, dtype=np.float64) if quad else np.asarray(R, dtype=op_dtype)

    def apply(vtop, vbot):
        """z = M_R^-1 v (u_R), then w = M_L^-1 Atilde_alpha z (u_A, u_L).  The top block of
        M_R^-1 and of M_L^-1 is I and Atilde_alpha's top-left block is alpha I: z_top = v_top
        enters w_top as alpha v_top, and only the products A z_bot and A^T z_top are
        rounded to u_A."""
        if quad:
            zh, zl = dd.solve_upper(Ro, vbot)
            wt, _ = dd.matvec(Ao, zh, zl, add=vtop, alpha=alpha)
            th, tl = dd.matvec_t(Ao, vtop)
            wb, _ = dd.solve_upper_t(Ro, th, tl)
            return zh.astype(wd), np.concatenate([wt, wb]).astype(wd)
        zb = solve_upper(Ro, vbot.astype(op_dtype)).astype(op_dtype)
        wt = alpha * vtop + (Ao @ zb).astype(wd)
        wb = solve_upper_t(Ro, (Ao.T @ vtop.astype(op_dtype)).astype(op_dtype)).astype(op_dtype)
        return zb.astype(wd), np.concatenate([wt, wb.astype(wd)])

    rhs = np.concatenate([np.asarray(f, np.float64), np.asarray(h, np.float64) / alpha]).astype(wd)
    beta = np.linalg.norm(rhs)
    info = dict(its=0, relres=0.0, converged=True)
    if beta == 0:
        return np.zeros(m), np.zeros(n), info
    V = np.zeros((m + n, maxit + 1), dtype=wd)
    Zb = np.zeros((n, maxit), dtype=wd)
    H = np.zeros((maxit + 1, maxit), dtype=wd)
    cs = np.zeros(maxit, dtype=wd)
    sn = np.zeros(maxit, dtype=wd)
    g = np.zeros(maxit + 1, dtype=wd)
    g[0] = beta
    V[:, 0] = rhs / beta
    k = 0
    relres = 1.0
    for j in range(maxit):
        Zb[:, j], w = apply(V[:m, j], V[m:, j])
        for i in range(j + 1):                 # modified Gram-Schmidt
            H[i, j] = np.dot(w, V[:, i])
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V[:, j + 1] = w / H[j + 1, j]
        for i in range(j):                     # previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        relres = abs(g[j + 1]) / beta
        if relres <= tol:
            break
    y = solve_upper(H[:k, :k], g[:k])
    dr = alpha * (V[:m, :k] @ y)
    dx = Zb[:, :k] @ y
    info.update(its=k, relres=float(relres), converged=bool(relres <= tol))
    return dr.astype(np.float64), dx.astype(np.float64), info
