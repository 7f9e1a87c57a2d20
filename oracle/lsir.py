"""Oracle: Algorithm 2 -- augmented-system LSIR with randomized preconditioning.

Test infrastructure only (see ``oracle/__init__.py``).

The steps, in the paper's order (Alg. 2, Sec. 4):
  - x_0 = LSQR(A, b) right-preconditioned by R, started at x_s       (u)
  - r_0 = b - A x_0                                                 (u)
  - then, for i = 0, 1, ... until the stopping rule holds:
      [f_i; g_i] = [b; 0] - [[I, A], [A^T, 0]] [r_i; x_i]             (u_r)
      h_i = R^-T g_i                                                 (u_r)
      FGMRES on M_L^-1 Atilde M_R^-1 [dr; dz] = [f_i; h_i], dx = R^-1 dz
                                                     (u, u_A, u_L, u_R)
      [r_{i+1}; x_{i+1}] = [r_i; x_i] + [dr; dx]                       (u)
Sec. 5: at most 30 refinement steps; FGMRES at most 50 iterations with the
LSQR tolerance; if the loop does not converge and kappa(A) < u_s^-1, the
loop is run again from (x_0, r_0) with u_A = u_L = u_R = u^2.

Stopping.  The paper stops when both forward errors against the true x*, r*
are <= 4u; ``lsir`` does exactly that when (xstar, rstar) are given.
Otherwise it uses a computable rule: stop after step i if
||dx_i|| <= u ||x_{i+1}|| and ||dr_i|| <= u ||r_{i+1}||, or if (i >= 1) the
contraction estimates rho = ||d_i|| / ||d_{i-1}|| are below 1/2 and
rho ||dx_i|| <= 4u ||x_{i+1}||, rho ||dr_i|| <= 4u ||r_{i+1}|| (the next
correction, i.e. the remaining error, is then within the 4u the paper asks
of the forward errors).

Here u_r is the correctly rounded residual of ``exact.residual_aug`` when
``ur='exact'`` and plain FP64 otherwise.  h_i = R^-T g_i: Alg. 2 marks this solve
with u_r, but Table 4's escalated rows (2*, 138* at kappa = 1e12 and 2*, 137* at
1e14) are reproduced only when h_i is solved in FP64 from the rounded g_i (2, 140
and 2, 141 here; a double-double solve from the double-double g_i gives 1, 71 and
2, 139).  The default reading is therefore the FP64 solve; ``h_ur=True`` (with
``ur='exact'``) takes the solve in double-double as Alg. 2 prints it
(``oracle.dd``), rounded to FP64 where FGMRES takes it.
"""
import numpy as np

from . import dd, exact
from .fgmres import fgmres
from .lsqr import lsqr
from .qr import solve_upper_t


def _residual(A, b, r, x, ur):
    if ur == "exact":
        return exact.residual_aug(A, b, r, x)
    f = b - r - A @ x
    g = -(A.T @ r)
    return f, g


def refine(A, b, R, x0, r0, u, tol, ir_maxit, gm_maxit, op_dtype, ur, xstar=None, rstar=None,
           gm_work_dtype=np.float64, alpha=1.0, h_ur=False):
    """The refinement loop of Alg. 2 from (x0, r0).  Returns (x, r, info).  ``alpha``
    scales the augmented system (Sec. 4.1; see ``fgmres``)."""
    x = np.array(x0, np.float64, copy=True)
    r = np.array(r0, np.float64, copy=True)
    its, gm_total, converged = 0, 0, False
    prev = None
    gm_its = []
    for _ in range(ir_maxit):
        f, g = _residual(A, b, r, x, ur)
        if ur == "exact" and h_ur:
            gh, gl = dd.matvec_t(A, -np.asarray(r, np.float64))   # g = -A^T r as double-double
            h = dd.solve_upper_t(np.asarray(R, np.float64), gh, gl)[0]
        else:
            h = solve_upper_t(R, g)
        dr, dx, ginfo = fgmres(A, R, f, h, tol, gm_maxit, op_dtype=op_dtype, work_dtype=gm_work_dtype,
                               alpha=alpha)
        x = x + dx
        r = r + dr
        its += 1
        gm_total += ginfo["its"]
        gm_its.append(ginfo["its"])
        if xstar is not None:
            ex, er = exact.forward_errors(x, r, xstar, rstar)
            done = ex <= 4 * u and er <= 4 * u
        else:
            ndx, ndr = np.linalg.norm(dx), np.linalg.norm(dr)
            nx, nr = np.linalg.norm(x), np.linalg.norm(r)
            done = ndx <= u * nx and ndr <= u * nr
            if not done and prev is not None:
                rx = ndx / prev[0] if prev[0] > 0 else 1.0
                rr = ndr / prev[1] if prev[1] > 0 else 1.0
                done = rx < 0.5 and rr < 0.5 and rx * ndx <= 4 * u * nx and rr * ndr <= 4 * u * nr
            prev = (ndx, ndr)
        if done:
            converged = True
            break
    return x, r, dict(its=its, gmres_total=gm_total, gmres_its=gm_its, converged=converged)


def lsir(A, b, R, xs, u, tol, lsqr_maxit=None, ir_maxit=30, gm_maxit=50,
         w_dtype=np.float64, op_dtype=None, ur="exact", us=None, kappa=None,
         xstar=None, rstar=None, escalate=True, gm_work_dtype=np.float64, alpha=1.0, h_ur=False):
    """Algorithm 2.  ``u`` is the unit roundoff of ``w_dtype``.

    Returns (x, r, info).  ``us`` (unit roundoff of the sketch) and ``kappa``
    drive the escalation rule of Sec. 5.  ``gm_work_dtype`` is the precision of
    FGMRES's basis, Gram-Schmidt and rotations (see ``fgmres``); the escalation
    raises only the products (u_A = u_L = u_R), as in Sec. 5: to double for u
    single (Table 3), to quad (double-double, ``oracle.dd``) with at most 80 FGMRES
    iterations for u double (Table 4).  ``alpha`` scales the augmented system
    (Sec. 4.1); ``h_ur`` solves h = R^-T g in u_r (see the module docstring).
    """
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    n = A.shape[1]
    if lsqr_maxit is None:
        lsqr_maxit = 2 * n
    if op_dtype is None:
        op_dtype = w_dtype
    x0, linfo = lsqr(A, b, R, xs, tol, lsqr_maxit, dtype=w_dtype)
    Aw = A.astype(w_dtype)
    r0 = (b.astype(w_dtype) - Aw @ x0.astype(w_dtype)).astype(np.float64)
    x0 = x0.astype(w_dtype).astype(np.float64)
    x, r, info = refine(A, b, R, x0, r0, u, tol, ir_maxit, gm_maxit, op_dtype, ur, xstar, rstar,
                        gm_work_dtype, alpha, h_ur)
    info["escalated"] = False
    if (not info["converged"] and escalate and us is not None and kappa is not None
            and kappa < 1.0 / us):
        double = np.dtype(w_dtype) == np.float64
        x, r, info = refine(A, b, R, x0, r0, u, tol, ir_maxit, max(gm_maxit, 80) if double else gm_maxit,
                            "dd" if double else np.float64, ur, xstar, rstar, gm_work_dtype, alpha, h_ur)
        info["escalated"] = True
    info["lsqr"] = linfo
    return x, r, info
