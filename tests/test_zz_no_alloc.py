"""lsq_qr_r_noalloc (QR in a fixed device scratch array, no allocation, no
handle) against lsq_qr_r on the same sketches, through the C ABI.

Collected last on purpose: it must pass both alone in a fresh process (first
call on the device does the scratch set-up) and after every other test.
"""
import numpy as np
import pytest
import torch

from conftest import dev, from_colmajor
from lsq_synth import randsvd_problem

pytestmark = pytest.mark.gpu

WORK_BYTES = 8388608      # LSQ_NOALLOC_WORK_BYTES
MAX_N = 1024              # LSQ_NOALLOC_MAX_N


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


def _sketch(lsq, handle, m, n, s, kappa, seed):
    P = randsvd_problem(m, n, kappa, rho=1e-2, seed=seed)
    A, b = dev(P.A), dev(P.b)
    Y = zeros(s * (n + 1))
    lsq.lsq_sketch(handle, A, b, m, n, s, "bf16", "f32", "f32", "f64", 1e-6, seed, None, Y)
    return A, b, Y


def _reference(lsq, handle, A, b, Y, m, n, s, up):
    R, xs = zeros(n * n), zeros(n)
    lsq.lsq_qr_r(handle, A, b, m, n, s, "bf16", up, "f32", "f64", 1e-6, 0, {"Y_in": Y}, R, xs)
    torch.cuda.synchronize()
    return from_colmajor(R, n, n), xs.cpu().numpy()


def _noalloc(lsq, Y, n, s, up):
    R, c = zeros(n * n), zeros(n)
    st = lsq.lsq_qr_r_noalloc(Y, s, n, up, R, c)
    assert st == 0
    return from_colmajor(R, n, n), c.cpu().numpy()


# (m, n, s, kappa): the first fits the FP32 blocked panel path, the last is the
# size of the m = 1e5, n = 500 workload's sketch (s = 4n), which fills most of
# the FP64 scratch (2000 * 501 * 8 bytes of 8 MiB).
CASES = [(5000, 130, 400, 1e2), (4000, 257, 600, 1e3), (8000, 500, 2000, 1e4)]


@pytest.mark.parametrize("up", ["f32", "f64"])
@pytest.mark.parametrize("m,n,s,kappa", CASES)
def test_noalloc_qr_matches_lsq_qr_r_twice(lsq, handle, up, m, n, s, kappa):
    A, b, Y = _sketch(lsq, handle, m, n, s, kappa, seed=n)
    R_ref, xs_ref = _reference(lsq, handle, A, b, Y, m, n, s, up)
    u = 2.0 ** -53 if up == "f64" else 2.0 ** -24
    nR = np.linalg.norm(R_ref, 2)
    outs = [_noalloc(lsq, Y, n, s, up) for _ in range(2)]     # two calls in a row
    for R, c in outs:
        assert np.all(np.isfinite(R)) and np.allclose(np.tril(R, -1), 0)
        # same kernels, same Y: equal to lsq_qr_r's R within a few ulps of ||R||
        assert np.linalg.norm(R - R_ref, 2) <= 8 * u * nR
        # c is Q^T Omega b: R^-1 c is lsq_qr_r's sketch-and-solve start x_s
        x = np.linalg.solve(np.triu(R), c)
        assert np.linalg.norm(x - xs_ref) <= 20 * n * kappa * u * np.linalg.norm(xs_ref)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_noalloc_sizes_beyond_scratch_are_rejected(lsq):
    Y, R, c = zeros(16), zeros(16), zeros(16)
    n = 500
    s_max64 = WORK_BYTES // 8 // (n + 1)
    assert lsq.lsq_qr_r_noalloc(Y, s_max64 + 1, n, "f64", R, c) == -9          # LSQ_E_SIZE
    assert lsq.lsq_qr_r_noalloc(Y, 2 * s_max64 + 2, n, "f32", R, c) == -9
    assert lsq.lsq_qr_r_noalloc(Y, 4 * (MAX_N + 1), MAX_N + 1, "f32", R, c) == -9
    with pytest.raises(lsq.LsqError):                                          # LSQ_E_INVAL
        lsq.lsq_qr_r_noalloc(Y, 10, 20, "f64", R, c)


def test_noalloc_rank_deficient_sketch(lsq, handle):
    m, n, s = 3000, 40, 160
    _, _, Y = _sketch(lsq, handle, m, n, s, 10.0, seed=3)
    Y.view(n + 1, s)[7].zero_()                                  # column 7 of Y is zero
    with pytest.raises(lsq.LsqError) as ei:
        lsq.lsq_qr_r_noalloc(Y, s, n, "f64", zeros(n * n), zeros(n))
    assert ei.value.status == -2                                 # LSQ_E_RANK
    # the scratch is usable again right after an error
    _, _, Y2 = _sketch(lsq, handle, m, n, s, 10.0, seed=4)
    R, c = _noalloc(lsq, Y2, n, s, "f64")
    assert np.all(np.diag(R) > 0)
