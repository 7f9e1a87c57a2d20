"""Generators for the synthetic least-squares inputs (see package docstring)."""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    A: np.ndarray            # m x n, FP64, C-contiguous (row-major)
    b: np.ndarray            # m, FP64
    sigma: np.ndarray        # singular values used to build A
    kappa: float
    x_true: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def n(self):
        return self.A.shape[1]


def _orthonormal_columns(rng, m, n):
    """m x n with orthonormal columns: CholeskyQR2 of a Gaussian matrix."""
    Q = rng.standard_normal((m, n))
    for _ in range(2):
        C = np.linalg.cholesky(Q.T @ Q)          # Q^T Q = C C^T
        Q = np.linalg.solve(C, Q.T).T            # Q C^-T
    return Q


def _haar(rng, n):
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]


def randsvd_problem(m, n, kappa, rho=1e-3, seed=0, kind="consistent+perp"):
    """A = U diag(sigma) V^T with geometric sigma from 1 to 1/kappa."""
    rng = np.random.default_rng(seed)
    U = _orthonormal_columns(rng, m, n)
    V = _haar(rng, n)
    if n > 1:
        sigma = float(kappa) ** (-np.arange(n) / (n - 1))
    else:
        sigma = np.ones(1)
    A = np.ascontiguousarray((U * sigma[None, :]) @ V.T)
    x_true = None
    if kind == "uniform":
        b = rng.uniform(0.0, 1.0, m)
        b /= np.linalg.norm(b)
    else:
        x_true = rng.standard_normal(n)
        ax = A @ x_true
        g = rng.standard_normal(m)
        for _ in range(2):
            g = g - U @ (U.T @ g)
        if rho > 0:
            # ||r||^2 / (||Ax||^2 + ||r||^2) = rho^2 (Ax and r orthogonal)
            g *= rho / np.sqrt(1 - rho * rho) * np.linalg.norm(ax) / np.linalg.norm(g)
        else:
            g[:] = 0
        b = ax + g
    return Problem(A=A, b=b, sigma=sigma, kappa=float(kappa), x_true=x_true,
                   meta=dict(m=m, n=n, kappa=kappa, rho=rho, seed=seed, kind=kind))


def paper_problem(kappa, m=1000, n=100, seed=0):
    """The Sec. 5 test shape: m = 1000, n = 100, b ~ U(0,1) normalised."""
    return randsvd_problem(m, n, kappa, seed=seed, kind="uniform")


def batch_specs(count=512, seed=0, m_range=(5000, 200000), n_range=(32, 256),
                kappa_range=(1e2, 1e8), rho_range=(1e-8, 1e-1)):
    """Shapes and conditioning of a batch of uneven problems (one dict each)."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        specs.append(dict(
            m=int(rng.integers(m_range[0], m_range[1] + 1)),
            n=int(rng.integers(n_range[0], n_range[1] + 1)),
            kappa=float(10 ** rng.uniform(np.log10(kappa_range[0]), np.log10(kappa_range[1]))),
            rho=float(10 ** rng.uniform(np.log10(rho_range[0]), np.log10(rho_range[1]))),
            seed=seed * 100003 + k + 1))
    return specs
