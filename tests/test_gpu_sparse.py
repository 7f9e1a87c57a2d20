"""The sparse sign sketch (Sec. 2; opts.sketch_kind = 1) through the C ABI against the oracle.

The sums are exact integers on per-column fixed-point grids on both sides, so the sketch
is compared bit for bit: over ragged column blocks of every shared-memory layout (4, 2 and
1 columns per CTA), several zeta, a row stride wider than n, and at m = 4e6 on sampled
columns (a column of Y depends only on that column of A, the row table and the largest
sketch-row count).  Then Algorithm 2 with the sparse sketch reaches the 4u level.
"""
import numpy as np
import pytest
import torch

from conftest import dev, from_colmajor
from lsq_synth import paper_problem, randsvd_problem
from oracle import exact, sparse

pytestmark = pytest.mark.gpu


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("m,n,s,zeta,lda", [(3000, 20, 80, 8, 0), (9000, 130, 520, 8, 0), (8000, 50, 7000, 3, 0),
                                            (20000, 10, 13000, 1, 0), (6000, 33, 140, 5, 40), (500, 1, 8, 8, 0)])
def test_sparse_sketch_is_bit_exact(lsq, handle, m, n, s, zeta, lda):
    P = randsvd_problem(m, n, 1e4, rho=1e-2, seed=m + n)
    A = P.A
    if lda:
        A = np.zeros((m, lda))
        A[:, :n] = P.A
    Y = zeros(s * (n + 1))
    opts = {"sketch_kind": 1, "sparse_zeta": zeta, "lda": lda}
    lsq.lsq_sketch(handle, dev(A), dev(P.b), m, n, s, "bf16", "f64", "f64", "f64", 1e-6, 17, opts, Y)
    ref = sparse.sparse_sketch(P.A, P.b, s, zeta, 17)
    got = from_colmajor(Y, s, n + 1)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_sparse_sketch_full_size_sampled_columns(lsq, handle):
    from lsq_synth.device import DeviceRandsvd
    m, n, s = 4_000_000, 1000, 4000
    gen = DeviceRandsvd(m, n, seed=4)
    A, b, _ = gen.problem(1e7, 1e-6)
    gen.release()
    Y = zeros(s * (n + 1))
    lsq.lsq_sketch(handle, A, b, m, n, s, "bf16", "f64", "f64", "f64", 1e-6, 3, {"sketch_kind": 1}, Y)
    cols = np.sort(np.random.default_rng(1).choice(n, 12, replace=False))
    As = A[:, torch.as_tensor(cols, device=A.device)].cpu().numpy()
    bs = b.cpu().numpy()
    ref = sparse.sparse_sketch(As, bs, s, 8, 3)          # the sampled columns and b
    got = Y.view(n + 1, s)[torch.as_tensor(np.append(cols, n), device=Y.device)].cpu().numpy().T
    assert np.array_equal(got, ref)
    del A, b, Y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_lsir_with_sparse_sketch_reaches_working_precision(lsq, handle, kappa):
    P = paper_problem(kappa, seed=8)
    m, n, s = 1000, 100, 400
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, s, "bf16", "f32", "f32", "f64", 1e-6, 0,
                            {"sketch_kind": 1}, x, r)
    xstar, rstar = exact.reference_solution(P.A, P.b)
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
    assert st == 0 and ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (ex, er)
    assert info.lsqr_its <= 25 and info.us_used == lsq.PREC["f64"]


def test_sparse_options_are_validated(lsq, handle):
    P = paper_problem(10.0, seed=1)
    Y = zeros(400 * 101)
    for bad in ({"sketch_kind": 2}, {"sketch_kind": 1, "sparse_zeta": 9}, {"sketch_kind": 1, "sparse_zeta": -1}):
        with pytest.raises(lsq.LsqError) as e:
            lsq.lsq_sketch(handle, dev(P.A), dev(P.b), 1000, 100, 400, "bf16", "f64", "f64", "f64", 1e-6, 0, bad, Y)
        assert e.value.status == -1
