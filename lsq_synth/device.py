"""The randsvd recipe of ``problems.randsvd_problem`` drawn on a CUDA device.

For the largest shapes (m up to 4e6, n = 1000) the host build takes minutes
and tens of GB of host memory, so the same construction -- U from CholeskyQR2
of a Gaussian m x n matrix, V Haar n x n, geometric sigma from 1 to 1/kappa,
b = A x_true + r_perp with r_perp orthogonal to range(U) -- runs here on the
device in FP64 with torch's seeded generator (a different stream than the
host generator's: same law, different draws).  U is kept so that several
kappa values share one draw; the factors sigma and V stay available, which
gives exact properties such as sigma(A R^-1) = sigma(Sigma V^T R^-1).

Only products and elementwise work run on the device: the n x n factorisations
(Cholesky of the Gram matrix, QR for V) run on the host with numpy, so the
generator needs no device linear-algebra library (torch loads its own lazily,
which fails under some profilers).
"""
import numpy as np


class DeviceRandsvd:
    def __init__(self, m, n, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.m, self.n = int(m), int(n)
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        Q = torch.randn(self.m, self.n, generator=g, device=device, dtype=torch.float64)
        for _ in range(2):                                   # CholeskyQR2: Q <- Q C^-T
            C = np.linalg.cholesky((Q.T @ Q).cpu().numpy())  # Q^T Q = C C^T (C well conditioned)
            CiT = torch.from_numpy(np.ascontiguousarray(np.linalg.inv(C).T)).to(device)
            Q = Q @ CiT
        self.U = Q
        Z = torch.randn(self.n, self.n, generator=g, device=device, dtype=torch.float64).cpu().numpy()
        V, Rz = np.linalg.qr(Z)
        V = V * np.where(np.diag(Rz) < 0, -1.0, 1.0)[None, :]
        self.V = torch.from_numpy(np.ascontiguousarray(V)).to(device)
        self.x_true = torch.randn(self.n, generator=g, device=device, dtype=torch.float64)
        gv = torch.randn(self.m, generator=g, device=device, dtype=torch.float64)
        for _ in range(2):
            gv = gv - self.U @ (self.U.T @ gv)
        self.perp = gv

    def sigma(self, kappa):
        n = self.n
        if n == 1:
            return np.ones(1)
        return float(kappa) ** (-np.arange(n) / (n - 1))

    def problem(self, kappa, rho, rows_per_chunk=1 << 18):
        """(A, b, r_perp) on the device: A = U diag(sigma) V^T (row-major FP64)."""
        torch = self.torch
        sig = torch.tensor(self.sigma(kappa), device=self.U.device, dtype=torch.float64)
        SVt = sig[:, None] * self.V.T
        A = torch.empty(self.m, self.n, device=self.U.device, dtype=torch.float64)
        for i0 in range(0, self.m, rows_per_chunk):
            i1 = min(self.m, i0 + rows_per_chunk)
            torch.matmul(self.U[i0:i1], SVt, out=A[i0:i1])
        ax = A @ self.x_true
        r = self.perp * (rho / np.sqrt(1.0 - rho * rho) * torch.linalg.norm(ax) / torch.linalg.norm(self.perp))
        return A, ax + r, r

    def release(self):
        self.U = None
        self.perp = None
