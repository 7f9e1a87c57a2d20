"""lsq_sketch (tcgen05 / CUDA-core) against the oracle's Algorithm 1 (the sketch)."""
import numpy as np
import pytest
import torch

from conftest import dev, from_colmajor
from lsq_synth import randsvd_problem
from oracle import rng, sketch

pytestmark = pytest.mark.gpu

FMTS = ["f16", "bf16", "e4m3", "bf16x3", "f32", "f64"]


def gpu_sketch(lsq, handle, A, b, s, fmt, seed, uw="f32", **opts):
    m, n = A.shape
    Y = torch.full((s * (n + 1),), float("nan"), dtype=torch.float64, device="cuda")
    lsq.lsq_sketch(handle, dev(A), dev(b), m, n, s, fmt, "f32", uw, "f64", 1e-6, seed, opts or None, Y)
    return from_colmajor(Y, s, n + 1)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("m,n,s", [(4133, 40, 200), (3100, 600, 640)])
def test_sketch_extracts_columns_exactly(lsq, handle, fmt, m, n, s):
    """With one-hot columns each Y entry is a single product: exact on both sides.  n = 600
    takes two column groups, whose CTAs share the generated operand (half each)."""
    r = np.random.default_rng(1)
    perm = r.choice(m, n + 1, replace=False)
    A = np.zeros((m, n))
    A[perm[:n], np.arange(n)] = 1.0
    b = np.zeros(m)
    b[perm[n]] = -1.0
    got = gpu_sketch(lsq, handle, A, b, s, fmt, 77)
    ref = sketch.sketch(A, b, s, 77, fmt)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("m,n,s", [(5000, 37, 150), (3001, 300, 320), (2100, 600, 640)])
def test_sketch_parity(lsq, handle, fmt, m, n, s):
    P = randsvd_problem(m, n, 1e3, rho=1e-2, seed=m + n)
    seed = 31 + n
    got = gpu_sketch(lsq, handle, P.A, P.b, s, fmt, seed)
    ref = sketch.sketch(P.A, P.b, s, seed, fmt)
    As, bs, kA, kb = sketch.cast_scaled(P.A, P.b, fmt)
    Gs = rng.sketch_operand(s, 0, m, seed, fmt)
    k = np.concatenate([kA, [kb]])
    mag = np.ldexp(np.abs(Gs) @ np.abs(np.column_stack([As, bs])), -k[None, :]) / np.sqrt(s)
    ulp = 2.0 ** -53 if fmt == "f64" else 2.0 ** -24   # accumulation precision
    err = np.abs(got - ref)
    # rigorous: every partial sum of m exact products rounds at most once per add
    assert np.all(err <= (m + 2) * ulp * mag + 1e-300)
    # typical: random-walk accumulation error, far below the worst case
    assert np.sqrt(np.mean((err / mag) ** 2)) <= 8 * np.sqrt(m) * ulp


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_sketch_no_colscale_matches_oracle_unscaled(lsq, handle, fmt):
    P = randsvd_problem(1500, 20, 10.0, seed=3)
    got = gpu_sketch(lsq, handle, P.A, P.b, 80, fmt, 5, no_colscale=1)
    Ab = np.column_stack([P.A, P.b])
    Gs = rng.sketch_operand(80, 0, 1500, 5, fmt)
    ref = Gs @ rng.round_to_format(Ab, fmt) / np.sqrt(80)
    mag = np.abs(Gs) @ np.abs(rng.round_to_format(Ab, fmt)) / np.sqrt(80)
    assert np.all(np.abs(got - ref) <= 1502 * 2.0 ** -24 * mag + 1e-300)


def test_sketch_full_size_sampled_entries(lsq, handle):
    """The bench workload (m=1e5, n=500, s=4n, BF16 and FP16): sampled entries vs the oracle."""
    m, n, s = 100000, 500, 2000
    P = randsvd_problem(m, n, 1e6, rho=1e-3, seed=1)
    for fmt in ("bf16", "f16", "bf16x3"):
        got = gpu_sketch(lsq, handle, P.A, P.b, s, fmt, 0)
        As, bs, kA, kb = sketch.cast_scaled(P.A, P.b, fmt)
        Ab = np.column_stack([As, bs])
        k = np.concatenate([kA, [kb]])
        r = np.random.default_rng(5)
        for i in r.choice(s, 6, replace=False):
            g = rng.round_to_format(rng.gaussian_block(int(i), int(i) + 1, 0, m, 0),
                                    rng.OPERAND_FORMAT[fmt])
            row = (g @ Ab)[0] / np.sqrt(s)
            ref = np.ldexp(row, -k)
            mag = np.ldexp((np.abs(g) @ np.abs(Ab))[0] / np.sqrt(s), -k)
            assert np.all(np.abs(got[i] - ref) <= (m + 2) * 2.0 ** -24 * mag)
            assert np.sqrt(np.mean(((got[i] - ref) / mag) ** 2)) <= 8 * np.sqrt(m) * 2.0 ** -24


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3", "bf16x3"])
@pytest.mark.parametrize("m,n,s", [(20000, 70, 256), (12000, 700, 768)])
def test_sketch_deferred_correction_matches_exact_mode(lsq, handle, fmt, m, n, s):
    """The GEMM on FP32 estimates plus the correction of near-midpoint entries gives the
    product with fl_s(G) itself: same values as resolving them inside the GEMM, up to the
    FP32 accumulation order, and bit-identical from run to run.  n = 700: two column
    groups sharing the generated operand, with the corrections read from both lists."""
    P = randsvd_problem(m, n, 1e3, rho=1e-2, seed=11)
    got = gpu_sketch(lsq, handle, P.A, P.b, s, fmt, 5)
    again = gpu_sketch(lsq, handle, P.A, P.b, s, fmt, 5)
    exact = gpu_sketch(lsq, handle, P.A, P.b, s, fmt, 5, sketch_exact=1)
    assert np.array_equal(got, again)
    As, bs, kA, kb = sketch.cast_scaled(P.A, P.b, fmt)
    Gs = rng.sketch_operand(s, 0, m, 5, fmt)
    k = np.concatenate([kA, [kb]])
    mag = np.ldexp(np.abs(Gs) @ np.abs(np.column_stack([As, bs])), -k[None, :]) / np.sqrt(s)
    assert np.all(np.abs(got - exact) <= 2 * (m + 2) * 2.0 ** -24 * mag + 1e-300)
    ref = sketch.sketch(P.A, P.b, s, 5, fmt)
    assert np.all(np.abs(got - ref) <= (m + 2) * 2.0 ** -24 * mag + 1e-300)


@pytest.mark.parametrize("m,n,s", [(5000, 37, 150), (9001, 300, 320)])
def test_bf16x3_cast_from_fp32_copy_is_bit_identical(lsq, handle, m, n, s):
    """The BF16X3 operand y = fl32(2^k x) formed from the FP32 working copy (u_w = F32: a
    power-of-two scaling of fl32(x) where that is exact) and from A alone (u_w = F64) is
    the same, so the sketches agree bit for bit.  The input has zeros, exact FP32 ties,
    columns whose FP32 copy is subnormal or overflows, and entries whose scaled value lands
    at the bottom of FP32's range (the copy is passed over there)."""
    P = randsvd_problem(m, n, 1e3, rho=1e-2, seed=21)
    A = P.A.copy()
    r = np.random.default_rng(3)
    A[r.random(A.shape) < 0.01] = 0.0
    A[:, 1] *= 2.0 ** -140                 # the FP32 copy of this column is subnormal
    A[:, 2] *= 2.0 ** 135                  # ... and here partly infinite
    A[::7, 3] *= 2.0 ** -136               # scaled entries near FP32's smallest normal
    A[::11, 4] = np.sign(A[::11, 4]) * (1.0 + 2.0 ** -24) * 2.0 ** -8   # ties of the FP32 rounding
    got32 = gpu_sketch(lsq, handle, A, P.b, s, "bf16x3", 9)
    got64 = gpu_sketch(lsq, handle, A, P.b, s, "bf16x3", 9, uw="f64")
    assert np.array_equal(got32, got64)
    ref = sketch.sketch(A, P.b, s, 9, "bf16x3")
    As, bs, kA, kb = sketch.cast_scaled(A, P.b, "bf16x3")
    Gs = rng.sketch_operand(s, 0, m, 9, "bf16x3")
    k = np.concatenate([kA, [kb]])
    mag = np.ldexp(np.abs(Gs) @ np.abs(np.column_stack([As, bs])), -k[None, :]) / np.sqrt(s)
    assert np.all(np.abs(got32 - ref) <= (m + 2) * 2.0 ** -24 * mag + 1e-300)
