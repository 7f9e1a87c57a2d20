"""The seeded input generators (lsq_synth) against the structure they promise.

The host generator feeds every oracle and parity test; the device generator
feeds the full-size tests, where only its invariants (not its draws) are
relied on.  Both are checked here on the CPU at small sizes.
"""
import numpy as np
import pytest
import torch

from lsq_synth import randsvd_problem
from lsq_synth.device import DeviceRandsvd


def _check_structure(A, b, r_perp, sigma, x_true, rho):
    # geometric singular values from 1 to 1/kappa
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sv, sigma, rtol=1e-12, atol=1e-15)
    # b = A x_true + r_perp with r_perp orthogonal to range(A) and ||r_perp|| = rho ||b||
    assert np.allclose(b, A @ x_true + r_perp, rtol=0, atol=1e-14 * np.linalg.norm(b))
    assert np.linalg.norm(A.T @ r_perp) <= 1e-13 * np.linalg.norm(r_perp)
    assert np.linalg.norm(r_perp) / np.linalg.norm(b) == pytest.approx(rho, rel=1e-12)


def test_host_randsvd_structure():
    P = randsvd_problem(700, 30, 1e4, rho=1e-3, seed=5)
    r_perp = P.b - P.A @ P.x_true
    _check_structure(P.A, P.b, r_perp, P.sigma, P.x_true, 1e-3)


@pytest.mark.parametrize("kappa,rho", [(1e3, 1e-2), (1e7, 1e-6)])
def test_device_randsvd_structure(kappa, rho):
    g = DeviceRandsvd(900, 24, seed=3, device="cpu")
    U = g.U.numpy()
    assert np.linalg.norm(U.T @ U - np.eye(24)) <= 1e-14
    V = g.V.numpy()
    assert np.linalg.norm(V.T @ V - np.eye(24)) <= 1e-14
    A, b, r = (t.numpy() for t in g.problem(kappa, rho, rows_per_chunk=256))
    _check_structure(A, b, r, g.sigma(kappa), g.x_true.numpy(), rho)


def test_device_randsvd_factors_give_sigma_of_A_Rinv():
    """sigma(A R^-1) = sigma(Sigma V^T R^-1) for any invertible R: the identity the
    full-size tests use to get kappa(A R^-1) without forming A R^-1."""
    g = DeviceRandsvd(500, 16, seed=8, device="cpu")
    A, _, _ = g.problem(1e3, 1e-2)
    R = np.triu(np.random.default_rng(1).standard_normal((16, 16))) + 4 * np.eye(16)
    direct = np.linalg.svd(np.linalg.solve(R.T, A.numpy().T).T, compute_uv=False)
    SVt = g.sigma(1e3)[:, None] * g.V.numpy().T
    via = np.linalg.svd(np.linalg.solve(R.T, SVt.T).T, compute_uv=False)
    assert np.allclose(direct, via, rtol=1e-11)


def test_device_randsvd_is_seeded():
    a = DeviceRandsvd(300, 8, seed=11, device="cpu").problem(10.0, 1e-2)[0]
    b = DeviceRandsvd(300, 8, seed=11, device="cpu").problem(10.0, 1e-2)[0]
    c = DeviceRandsvd(300, 8, seed=12, device="cpu").problem(10.0, 1e-2)[0]
    assert torch.equal(a, b) and not torch.equal(a, c)
