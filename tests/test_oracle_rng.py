"""Pins for the oracle's sketch-matrix generator (Philox + FP64 Box-Muller + rounding)."""
import numpy as np
import pytest
from fractions import Fraction

from oracle import rng

mp = pytest.importorskip("mpmath")


def test_philox_known_answers(golden):
    for row in golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = rng.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_is_vectorised_consistently():
    c0 = np.arange(100, dtype=np.uint64)
    out = rng.philox4x32_10(c0, 7, 0, 0, 11, 13)
    for k in (0, 17, 99):
        single = rng.philox4x32_10(int(c0[k]), 7, 0, 0, 11, 13)
        assert [int(o[k]) for o in out] == [int(s) for s in single]


def _edge_words():
    r = np.random.default_rng(5)
    w = r.integers(0, 2 ** 32, 1500, dtype=np.uint64)
    edges = [0, 1, 2, 3, 2 ** 29 - 1, 2 ** 29, 2 ** 30 - 1, 2 ** 30, 2 ** 31 - 1, 2 ** 31,
             3 * 2 ** 30, 0xB504F333, 0xB504F334, 2 ** 32 - 1000, 2 ** 32 - 2, 2 ** 32 - 1]
    return np.concatenate([w, np.array(edges, dtype=np.uint64)])


def test_ln_u1_within_two_ulps_of_exact():
    mp.mp.prec = 120
    a = _edge_words()
    got = rng.ln_u1(a)
    for ai, gi in zip(a, got):
        exact = mp.log(mp.mpf(int(ai) + 1) / 2 ** 32)
        if exact == 0:
            assert gi == 0.0
            continue
        assert abs((mp.mpf(gi) - exact) / exact) <= 2 * 2.0 ** -53


def test_cos_sin_2pi_within_two_ulps_of_exact():
    mp.mp.prec = 120
    b = _edge_words()
    c, s = rng.cos_sin_2pi(b)
    for bi, ci, si in zip(b, c, s):
        th = 2 * mp.pi * mp.mpf(int(bi)) / 2 ** 32
        assert abs(mp.mpf(ci) - mp.cos(th)) <= 2 * 2.0 ** -53
        assert abs(mp.mpf(si) - mp.sin(th)) <= 2 * 2.0 ** -53
    # exact special angles: quadrant boundaries
    c, s = rng.cos_sin_2pi(np.array([0, 2 ** 30, 2 ** 31, 3 * 2 ** 30], dtype=np.uint64))
    assert list(c) == [1.0, 0.0, -1.0, 0.0] or np.allclose(c, [1, 0, -1, 0], atol=0)
    assert np.array_equal(np.abs(s), [0.0, 1.0, 0.0, 1.0])


def test_gaussian_moments_and_ks():
    stats = pytest.importorskip("scipy.stats")
    G = rng.gaussian_block(0, 64, 0, 8192, seed=3).ravel()
    n = G.size
    assert abs(G.mean()) < 5 / np.sqrt(n)
    assert abs(G.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(G ** 4) - 3) < 5 * np.sqrt(96 / n)
    assert stats.kstest(G, "norm").pvalue > 1e-4
    # rows and columns are independent streams: no correlation between neighbours
    Gm = rng.gaussian_block(0, 256, 0, 2048, seed=3)
    assert abs(np.mean(Gm[:, :-1] * Gm[:, 1:])) < 5 / np.sqrt(Gm.size)
    assert abs(np.mean(Gm[:-1, :] * Gm[1:, :])) < 5 / np.sqrt(Gm.size)


def test_gaussian_block_is_a_pure_function_of_indices():
    full = rng.gaussian_block(0, 12, 0, 37, seed=2 ** 40 + 5)
    part = rng.gaussian_block(5, 9, 13, 30, seed=2 ** 40 + 5)
    assert np.array_equal(full[5:9, 13:30], part)
    other = rng.gaussian_block(0, 12, 0, 37, seed=2 ** 40 + 6)
    assert not np.array_equal(full, other)


def test_gaussian_pair_matches_box_muller_definition():
    mp.mp.prec = 100
    a = np.array([5, 2 ** 31 + 7, 2 ** 32 - 5], dtype=np.uint64)
    b = np.array([123456789, 2 ** 31 + 1, 4000000000], dtype=np.uint64)
    ge, go = rng.gaussian_pair(a, b)
    for k in range(3):
        u1 = mp.mpf(int(a[k]) + 1) / 2 ** 32
        u2 = mp.mpf(int(b[k])) / 2 ** 32
        r = mp.sqrt(-2 * mp.log(u1))
        assert abs(ge[k] - r * mp.cos(2 * mp.pi * u2)) <= 8 * 2.0 ** -53 * max(1, abs(ge[k]))
        assert abs(go[k] - r * mp.sin(2 * mp.pi * u2)) <= 8 * 2.0 ** -53 * max(1, abs(go[k]))
    ge, go = rng.gaussian_pair(np.array([2 ** 32 - 1], dtype=np.uint64), np.array([7], dtype=np.uint64))
    assert ge[0] == 0.0 and go[0] == 0.0 and not np.signbit(ge[0])


def _exact_round(x, fmt):
    """Brute-force nearest-even rounding with exact rationals (small samples)."""
    mbits, emin, xmax, sat = rng.FORMATS[fmt]
    xf = Fraction(float(x))
    if xf == 0:
        return 0.0
    sgn = 1 if xf > 0 else -1
    ax = abs(xf)
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    while Fraction(2) ** e > ax:
        e -= 1
    while Fraction(2) ** (e + 1) <= ax:
        e += 1
    q = max(e, emin) - mbits
    y = ax / Fraction(2) ** q
    fl = y.numerator // y.denominator
    rem = y - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = float(Fraction(fl) * Fraction(2) ** q)
    if val > xmax:
        val = xmax if sat else float("inf")
    return sgn * val


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3", "f32"])
def test_round_to_format_matches_exact_rational_rounding(fmt):
    r = np.random.default_rng(9)
    x = np.concatenate([r.standard_normal(400) * 3, r.standard_normal(100) * 1e-5,
                        r.standard_normal(50) * 1e-9, [0.0, -0.0, 500.0, -1e6]])
    got = rng.round_to_format(x, fmt)
    for xi, gi in zip(x, got):
        assert gi == _exact_round(xi, fmt), (fmt, xi, gi)


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3"])
def test_round_to_format_ties_go_to_even(fmt):
    mbits, emin, _, _ = rng.FORMATS[fmt]
    one_ulp = 2.0 ** -mbits
    mid_even = 1.0 + 0.5 * one_ulp         # between 1 (even) and 1 + ulp (odd)
    mid_odd = 1.0 + 1.5 * one_ulp          # between 1 + ulp (odd) and 1 + 2ulp (even)
    got = rng.round_to_format(np.array([mid_even, mid_odd, -mid_even]), fmt)
    assert list(got) == [1.0, 1.0 + 2 * one_ulp, -1.0]


def test_round_to_format_agrees_with_library_conversions():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(4)
    x32 = (r.standard_normal(20000) * np.exp(r.uniform(-8, 8, 20000))).astype(np.float32)
    x = x32.astype(np.float64)              # exact, so no double rounding in the libraries
    assert np.array_equal(rng.round_to_format(x, "f16"), x32.astype(np.float16).astype(np.float64))
    t = torch.from_numpy(x32)
    assert np.array_equal(rng.round_to_format(x, "bf16"), t.to(torch.bfloat16).double().numpy())
    xs = np.clip(x32, -440, 440)
    ts = torch.from_numpy(xs)
    assert np.array_equal(rng.round_to_format(xs.astype(np.float64), "e4m3"),
                          ts.to(torch.float8_e4m3fn).double().numpy())
    assert rng.round_to_format(np.array([1e4, -1e4]), "e4m3").tolist() == [448.0, -448.0]
