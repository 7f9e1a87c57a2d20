"""Seeded synthetic least-squares problems shaped like the paper's workloads.

This module holds input generation only -- none of the solver's arithmetic --
and is the one piece shared by the CPU oracle's tests and the CUDA path's
tests and benchmark.

The paper's experiments (Sec. 5) use MATLAB ``gallery('randsvd', [m, n],
kappa, 3)`` matrices: geometrically distributed singular values with random
orthogonal factors.  This generator builds matrices with that structure from
its own seeded normal draws (numpy PCG64), not from MATLAB's code:

    A = U diag(sigma) V^T,  sigma_i = kappa^(-(i-1)/(n-1))  (sigma_1 = 1),
    U: m x n with orthonormal columns (CholeskyQR2 of a Gaussian matrix),
    V: n x n Haar orthogonal (QR of a Gaussian matrix, R-diagonal signs fixed).

Right-hand sides:
* ``kind='consistent+perp'``: b = A x_true + r_perp with x_true ~ N(0, I),
  r_perp = (I - U U^T) g scaled so that ||r_perp|| / ||b|| = rho.
* ``kind='uniform'``: b ~ U(0, 1) normalised to unit norm (Sec. 5).

The largest shapes are drawn on the device instead (``device.DeviceRandsvd``,
same construction, torch's seeded generator).
"""
from .problems import Problem, randsvd_problem, paper_problem, batch_specs  # noqa: F401
