"""Oracle: closed forms from the paper and from random-matrix theory, used as pins.

Test infrastructure only (see ``oracle/__init__.py``).

* Sec. 2: for Omega A = Q P with orthonormal Q, kappa(A P^-1) = kappa(Omega U)
  and ||A P^-1|| = ||(Omega U)^+|| (U = left singular vectors of A).
* Eq. (4.1): kappa of [[alpha I, A R^-1], [R^-T A^T, 0]] from the extreme
  singular values of A R^-1.
* Unscaled augmented matrix [[I, A], [A^T, 0]]: eigenvalues 1 (m - n times)
  and 1/2 +- sqrt(1/4 + sigma_i^2).
* Marchenko-Pastur: an s x n matrix with i.i.d. N(0, 1/s) entries has
  singular values filling [1 - sqrt(n/s), 1 + sqrt(n/s)] as n, s grow with
  n/s fixed; Omega U is such a matrix for Gaussian Omega.
"""
import numpy as np


def kappa_prec_aug(alpha, smax, smin):
    """Sec. 4.1: kappa(M_L^-1 Atilde_alpha M_R^-1) from the extreme singular values of
    A R^-1.  The eigenvalues of [[alpha I, B], [B^T, 0]] (B = A R^-1, m > n) are alpha
    (m - n times) and (alpha +- sqrt(alpha^2 + 4 sigma_i^2)) / 2, so the smallest
    magnitude is min(alpha, (sqrt(alpha^2 + 4 sigma_min^2) - alpha) / 2).  The printed
    formula has min{2, ...} in the denominator, which is this one at alpha = 1 (the only
    value Sec. 5 uses); the 2 alpha here is the reading for alpha != 1."""
    num = alpha + np.sqrt(alpha ** 2 + 4 * smax ** 2)
    den = min(2.0 * alpha, np.sqrt(alpha ** 2 + 4 * smin ** 2) - alpha)
    return num / den


def kappa_prec_aug_bound(norm_ar, norm_ar_pinv):
    """Eq. (4.2): bound on the unscaled (alpha = 1) preconditioned kappa."""
    if norm_ar_pinv <= 1 / np.sqrt(2):
        return 1 + norm_ar
    return (2 + 2 * norm_ar) / (np.sqrt(1 + 4 / norm_ar_pinv ** 2) - 1)


def kappa_aug(smax, smin):
    """kappa([[I, A], [A^T, 0]]) for A with extreme singular values smax, smin."""
    lam_max = 0.5 + np.sqrt(0.25 + smax ** 2)
    lam_min = min(1.0, np.sqrt(0.25 + smin ** 2) - 0.5)
    return lam_max / lam_min


def mp_limits(n, s):
    """Marchenko-Pastur limits of (||A R^-1||, ||(A R^-1)^+||, kappa(A R^-1))."""
    t = np.sqrt(n / s)
    return 1 / (1 - t), 1 + t, (1 + t) / (1 - t)


def dense_matrix(op, nrows, ncols):
    """Materialise a linear operator column by column (small cases only)."""
    M = np.zeros((nrows, ncols))
    for j in range(ncols):
        e = np.zeros(ncols)
        e[j] = 1.0
        M[:, j] = op(e)
    return M
