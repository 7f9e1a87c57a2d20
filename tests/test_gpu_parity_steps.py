"""Stage-level parity through the C ABI against the oracle (Algorithm 2), on the same inputs.

* One refinement step (lsq_ir_step: FP64 residuals, h = R^-T g, FGMRES, update) against
  ``oracle.lsir.refine`` with one step and the same R, x_0, r_0: the same number of
  FGMRES iterations and the same correction.  The correction is compared in the
  variables FGMRES works in, [dr; R dx] (Eq. 1.2 with M_R = diag(I, R)).  GMRES is
  backward stable, so after k iterations each side's iterate is within about
  k kappa_p u_A of the exact-arithmetic one, kappa_p = kappa(M_L^-1 Atilde M_R^-1)
  (Eq. 4.1, from the extreme singular values of A R^-1); the preconditioner M_R^-1
  itself is a triangular solve in u_R = u_A, whose forward error is up to kappa(R) u_A
  (the u_R kappa(A) terms of the paper's analysis).  The bound below is
  20 (k kappa_p + kappa(R)) u_A, plus the FGMRES tolerance when the iteration counts
  differ by one.
* FP32 LSQR (Algorithm 2, LSQR start) with the oracle's R and start, both sides run
  for the same number of iterations: elementwise, the GPU's iterate is no farther from
  the FP64 iterate of the same k steps than four times the oracle's FP32 iterate is.
* lsq_lsir_host returns bit for bit what lsq_lsir returns on the same data.
* Every problem of a batched call against the oracle's reference solution (4u).
"""
import functools

import numpy as np
import pytest
import torch

from conftest import colmajor, dev
from lsq_synth import randsvd_problem
from oracle import exact, lsir, lsqr, qr, sketch, theory

pytestmark = pytest.mark.gpu


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=2)
def _setup(m, n, kappa, seed):
    P = randsvd_problem(m, n, kappa, rho=1e-3, seed=seed)
    s = 4 * n
    Y = sketch.sketch(P.A, P.b, s, 5, "f64")
    R, c = qr.householder_qr(Y, n)
    x0 = qr.sketch_and_solve(R, c)
    r0 = P.b - P.A @ x0
    sv = np.linalg.svd(P.A @ np.linalg.inv(R), compute_uv=False)
    return P, s, R, x0, r0, sv


@pytest.mark.parametrize("uw,kappa,arnoldi,m,n", [
    ("f64", 1e3, 1, 3000, 60), ("f64", 1e6, 1, 3000, 60), ("f32", 1e3, 1, 3000, 60), ("f32", 1e5, 1, 3000, 60),
    ("f64", 1e6, 2, 3000, 60), ("f32", 1e5, 2, 3000, 60), ("f64", 1e5, 2, 400000, 40),
    ("f32", 1e5, 2, 400000, 40), ("f64", 1e6, 3, 3000, 60), ("f32", 1e5, 3, 400000, 40),
    ("f64", 1e4, 1, 4000, 1000), ("f32", 1e4, 1, 4000, 1000)])
def test_refinement_step_matches_oracle(lsq, handle, uw, kappa, arnoldi, m, n):
    """arnoldi = 1: classical Gram-Schmidt with the selective second pass; 2: modified
    Gram-Schmidt (the oracle's form) with the work vector in shared memory; 3: the same
    with it in global memory (m = 4e5 runs the unrolled row loop).  n = 1000: the
    triangular solves run on the cluster with streamed tiles."""
    P, s, R, x0, r0, sv = _setup(m, n, kappa, seed=11)
    tol = 1e-10 if uw == "f64" else 1e-6
    ua = 2.0 ** -53 if uw == "f64" else 2.0 ** -24
    dt = np.float64 if uw == "f64" else np.float32
    xo, ro, io = lsir.refine(P.A, P.b, R, x0, r0, ua, tol, 1, 50, dt, "f64")
    x, r = dev(x0), dev(r0)
    st, info = lsq.lsq_ir_step(handle, dev(P.A), dev(P.b), m, n, s, "f64", "f64", uw, "f64", tol, 5,
                               {"gmres_maxit": 50, "arnoldi": arnoldi}, dev(colmajor(R)), x, r)
    kg, ko = info.gmres_its[0], io["gmres_its"][0]
    assert st == (0 if info.gmres_relres[0] <= tol else 1)
    assert abs(kg - ko) <= (0 if uw == "f64" else 1), (kg, ko)
    dxg, drg = x.cpu().numpy() - x0, r.cpu().numpy() - r0
    dxo, dro = xo - x0, ro - r0
    kp = theory.kappa_prec_aug(1.0, sv[0], sv[-1])
    bound = 20 * (max(kg, ko) * kp + np.linalg.cond(R)) * ua + (tol * kp if kg != ko else 0.0)
    # [dr; R dx]: the FGMRES correction in its own variables
    dg = np.concatenate([drg, R @ dxg])
    do = np.concatenate([dro, R @ dxo])
    rel = np.linalg.norm(dg - do) / np.linalg.norm(do)
    print(uw, kappa, arnoldi, m, "its", kg, ko, "kappa_p", kp, "rel", rel, "bound", bound)
    assert rel <= bound, (rel, bound)
    # the updated residual and solution themselves
    assert np.linalg.norm(r.cpu().numpy() - ro) <= bound * np.linalg.norm(do) + 1e-300


@pytest.mark.parametrize("m,n,kappa", [(3000, 60, 1e2), (2500, 130, 1e4), (4000, 200, 1e6), (3500, 760, 1e3),
                                       (4000, 1000, 1e4)])
def test_fp32_lsqr_iterates_elementwise(lsq, handle, m, n, kappa):
    """Both sides take exactly k FP32 iterations (tol 0) from the oracle's x_s with the
    oracle's R; the oracle's FP64 LSQR with the same R, start and k is the yardstick.
    Elementwise, |x_gpu - x_64| <= 4 max(|x_or32 - x_64|_inf) (the GPU's FP32 LSQR is at
    least as accurate as the oracle's, within a factor of four)."""
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=3)
    s = 4 * n
    Y = sketch.sketch(P.A, P.b, s, 1, "f32")
    R, c = qr.householder_qr(Y, n, dtype=np.float32)
    xs = qr.sketch_and_solve(R, c)
    k = 12
    x_or, info_or = lsqr.lsqr(P.A, P.b, R, xs, 0.0, k, dtype=np.float32)
    x_64, _ = lsqr.lsqr(P.A, P.b, R, xs, 0.0, k, dtype=np.float64)
    x = zeros(n)
    st, info = lsq.lsq_lsqr(handle, dev(P.A), dev(P.b), m, n, s, "f32", "f32", "f32", "f64", 1e-30, 1,
                            {"R_in": dev(colmajor(R)), "x0_in": dev(xs), "lsqr_maxit": k}, x)
    assert info.lsqr_its == info_or["its"] == k
    e_or = np.max(np.abs(x_or - x_64))
    e_gpu = np.abs(x.cpu().numpy() - x_64)
    print(m, n, kappa, "gpu", np.max(e_gpu), "oracle32", e_or, "x", np.max(np.abs(x_64)))
    assert np.all(e_gpu <= 4 * e_or), (np.max(e_gpu), e_or)


def test_lsir_host_is_bit_equal_to_device_solve(lsq, handle):
    m, n, s = 5000, 80, 320
    P = randsvd_problem(m, n, 1e4, rho=1e-3, seed=21)
    xd, rd = zeros(n), zeros(m)
    std, infod = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "bf16x3", "f32", "f32", "f64", 1e-6, 7,
                              None, xd, rd)
    hA = torch.from_numpy(P.A).pin_memory()
    hb = torch.from_numpy(P.b).pin_memory()
    hx = torch.zeros(n, dtype=torch.float64).pin_memory()
    hr = torch.zeros(m, dtype=torch.float64).pin_memory()
    sth, infoh = lsq.lsq_lsir_host(handle, hA, hb, m, n, s, "bf16x3", "f32", "f32", "f64", 1e-6, 7, None, hx, hr)
    assert std == sth == 0
    assert torch.equal(hx, xd.cpu()) and torch.equal(hr, rd.cpu())
    assert infoh.gmres_its_total == infod.gmres_its_total and infoh.lsqr_its == infod.lsqr_its
    # numpy arrays (pageable host memory) take the same path
    x2, r2 = np.zeros(n), np.zeros(m)
    lsq.lsq_lsir_host(handle, P.A, P.b, m, n, s, "bf16x3", "f32", "f32", "f64", 1e-6, 7, None, x2, r2)
    assert np.array_equal(x2, hx.numpy()) and np.array_equal(r2, hr.numpy())


def test_batched_problems_reach_the_oracle_solution(lsq, handle):
    """Each problem of one lsq_lsir_batched call (uneven m, n, kappa, rho) against the
    oracle's reference solution: forward errors in x and r within 4u (Sec. 5)."""
    shapes = [(3000, 32, 1e2, 1e-1), (7000, 64, 1e4, 1e-4), (5000, 100, 1e3, 1e-6), (4100, 45, 10.0, 1e-2),
              (9000, 77, 1e5, 1e-3), (6500, 128, 1e6, 1e-5)]
    probs, Ps = [], []
    for k, (m, n, kappa, rho) in enumerate(shapes):
        P = randsvd_problem(m, n, kappa, rho=rho, seed=60 + k)
        Ps.append(P)
        probs.append(dict(A=dev(P.A), b=dev(P.b), m=m, n=n, s=4 * n, seed=k, x=zeros(n), r=zeros(m)))
    st, sts, infos = lsq.lsq_lsir_batched(handle, probs, "bf16x3", "f32", "f32", "f64", 1e-6)
    assert st == 0 and all(v == 0 for v in sts)
    u = 2.0 ** -24
    for P, pr, inf in zip(Ps, probs, infos):
        xstar, rstar = exact.reference_solution(P.A, P.b)
        ex, er = exact.forward_errors(pr["x"].cpu().numpy(), pr["r"].cpu().numpy(), xstar, rstar)
        assert inf.ir_converged == 1 and ex <= 4 * u and er <= 4 * u, (P.meta, ex, er)
