"""Integer rounding of the cast pass (csrc/cast.cuh) against the oracle.

The cast A_s = fl_s(2^k A) of Sec. 3.2 runs on integer units on the GPU.  A
host build of the same header is compared bit for bit with
``oracle.rng.round_to_format`` (FP32: numpy's conversion) on random, sparse-bit
(tie-heavy) and range-edge inputs; the integer path may decline (then the
kernel uses the FP64 definition) only where the result leaves the format's
normal range or the input is subnormal or non-finite.  The BF16X3 operand (the
three BF16 terms of y = fl32(2^k A)) is compared with the oracle's cast for
every finite input, through the FP32 copy's power-of-two scaling where that
is exact and through the FP64 value elsewhere.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06319_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "native", "cast_harness.cpp")

# format -> (fraction bits, min normal exponent, max exponent handled, width)
ENC = {"bf16": (7, -126, 127, 16), "f16": (10, -14, 15, 16), "e4m3": (3, -6, 7, 8),
       "f32": (23, -126, 127, 32)}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("cast") / "cast_harness")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, HARNESS, "-o", exe], check=True)
    return exe


def run(exe, fmt, u, k):
    lines = [fmt] + [f"{int(a):x} {int(b)}" for a, b in zip(u, k)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    res = np.array([[int(w, 16) if i else int(w) for i, w in enumerate(l.split())]
                    for l in out.stdout.strip().splitlines()], dtype=np.int64)
    return res[:, 0].astype(bool), res[:, 1:].astype(np.uint32)


def inputs(seed, fmt):
    """FP64 bit patterns and exponents k: random, sparse-bit and edge cases."""
    r = np.random.default_rng(seed)
    mb, emin, emax, _ = ENC["f32" if fmt == "bf16x3" else fmt]
    n = 6000
    sign = r.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    E = r.integers(1023 - 30, 1023 + 30, n).astype(np.uint64)
    frac = r.integers(0, 2 ** 52, n, dtype=np.uint64)
    u_rand = sign | (E << np.uint64(52)) | frac
    # sparse significands: a few set bits -> many exact ties at every term
    sp = np.zeros(n, dtype=np.uint64)
    for _ in range(4):
        sp |= np.uint64(1) << r.integers(0, 52, n).astype(np.uint64)
    u_sparse = sign | (E << np.uint64(52)) | sp
    # all-ones significands: rounding carries into the next binade
    u_ones = sign[:200] | (E[:200] << np.uint64(52)) | np.uint64(2 ** 52 - 1)
    k = r.integers(-12, 13, 2 * n + 200)
    u = np.concatenate([u_rand, u_sparse, u_ones])
    # edges of the format's range: 2^k x around 2^emin and 2^(emax+1)
    edge_vals, edge_k = [], []
    for e in (emin - 1, emin, emax, emax + 1):
        x = np.ldexp(1.0 + r.random(300), e) * np.where(r.random(300) < 0.5, -1.0, 1.0)
        edge_vals.append(x)
        edge_k.append(np.zeros(300, dtype=np.int64))
    specials = np.array([0.0, -0.0, 5e-324, -2.2250738585072014e-308, np.inf, -np.inf, np.nan, 1.0, -1.0])
    xs = np.concatenate(edge_vals + [specials])
    u = np.concatenate([u, xs.view(np.uint64)])
    k = np.concatenate([k] + edge_k + [np.zeros(len(specials), dtype=np.int64)])
    return u, k


def bits_of(vals, fmt):
    """Bit patterns of values representable in fmt (normal range or zero)."""
    v = np.asarray(vals, dtype=np.float64)
    if fmt == "f32":
        return v.astype(np.float32).view(np.uint32).astype(np.uint32)
    if fmt == "bf16":
        return (v.astype(np.float32).view(np.uint32) >> 16).astype(np.uint32)
    if fmt == "f16":
        return v.astype(np.float16).view(np.uint16).astype(np.uint32)
    # e4m3: sign | (exponent + 7) << 3 | fraction, normal values and zeros
    mb, _, _, w = ENC[fmt]
    out = np.zeros(v.shape, dtype=np.uint32)
    nz = v != 0
    f, ex = np.frexp(np.abs(v[nz]))
    lead = ex - 1
    mant = np.rint((np.abs(v[nz]) / np.ldexp(1.0, lead) - 1.0) * 2 ** mb).astype(np.uint32)
    out[nz] = ((lead + 7).astype(np.uint32) << mb) | mant
    out |= (np.signbit(v).astype(np.uint32) << (w - 1))
    return out


def in_normal_range(vals, fmt):
    mb, emin, emax, _ = ENC[fmt]
    v = np.asarray(vals, dtype=np.float64)
    _, ex = np.frexp(np.abs(v))
    lead = ex - 1
    return (v == 0) | (np.isfinite(v) & (lead >= emin) & (lead <= emax))


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3", "f32"])
def test_integer_cast_matches_oracle_rounding(harness, fmt):
    u, k = inputs(11, fmt)
    ok, t = run(harness, fmt, u, k)
    x = u.view(np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        v = np.ldexp(x, k)
    base = fmt
    finite_in = np.isfinite(x) & ((x == 0) | (np.abs(x) >= 2.2250738585072014e-308))
    if fmt == "f32":
        with np.errstate(over="ignore"):
            terms = [v.astype(np.float32).astype(np.float64)]
    else:
        terms = [rng.round_to_format(np.where(finite_in, v, 0.0), fmt)]
    expect_ok = finite_in.copy()
    for tv in terms:
        expect_ok &= in_normal_range(tv, base)
    # the values each term rounds (exact differences in FP64)
    vin = np.where(finite_in, v, 0.0)
    with np.errstate(invalid="ignore"):
        raw = [vin] if len(terms) == 1 else [vin, vin - terms[0], vin - terms[0] - terms[1]]
    emin = ENC[base][1]
    below = np.zeros(len(u), dtype=bool)
    for rv in raw:
        below |= (rv != 0) & (np.abs(rv) < np.ldexp(1.0, emin))
    # never accepts where the FP64 definition is needed; declines otherwise only
    # for values below the normal range before rounding (their result may still
    # round to a normal number or to zero)
    assert not np.any(ok & ~expect_ok), np.flatnonzero(ok & ~expect_ok)[:10]
    assert not np.any(~ok & expect_ok & ~below), np.flatnonzero(~ok & expect_ok & ~below)[:10]
    for i, tv in enumerate(terms):
        want = bits_of(np.where(ok, tv, 0.0), base)
        assert np.array_equal(t[ok, i], want[ok]), (i, np.flatnonzero(t[ok, i] != want[ok])[:10])
    assert not np.any(t[:, 1:])
    # the integer path covers (almost) everything a scaled cast sees: values of
    # magnitude up to 2^(t+1) whose terms stay far above the normal range's floor
    if base in ("bf16", "f32"):
        assert ok[:12200].mean() > 0.99
    else:
        assert ok[:12200].sum() > 1000


def test_bf16x3_terms_match_oracle_cast(harness):
    """Every finite input, including values whose scaled FP32 rounding is subnormal or
    near the bottom of the normal range (there the header leaves the FP32 copy and
    rounds the FP64 value): the three terms are the oracle's split of fl32(2^k x)."""
    u, k = inputs(12, "bf16x3")
    # scalings that push entries to the bottom of FP32's range and below it
    r = np.random.default_rng(13)
    xs = np.ldexp(1.0 + r.random(3000), r.integers(-160, -110, 3000)) * np.where(r.random(3000) < 0.5, -1, 1)
    u = np.concatenate([u, xs.view(np.uint64)])
    k = np.concatenate([k, r.integers(-12, 13, 3000)])
    x = u.view(np.float64)
    keep = np.isfinite(x)
    u, k, x = u[keep], k[keep], x[keep]
    fast, t = run(harness, "bf16x3", u, k)
    with np.errstate(over="ignore"):
        y = rng.round_to_format(np.ldexp(x, k), "f32")
    small = np.abs(y) < 2.0 ** 127   # edge values whose hi term overflows BF16 are left out
    terms = rng.split3(np.where(small, y, 0.0), "bf16")
    for i, tv in enumerate(terms):
        want = (tv.astype(np.float32).view(np.uint32) >> 16).astype(np.uint32)
        assert np.array_equal(t[small, i], want[small]), (i, np.flatnonzero(t[small, i] != want[small])[:10])
    # the FP32 copy's scaling carries the bulk of a column's entries
    assert fast[:12200].mean() > 0.99
    assert not np.all(fast[-3000:])


def test_one_add_fp32_rounding_matches_numpy(harness):
    """The column-max pass's FP64 -> FP32 rounding (one 64-bit add at bit 29, then an
    exponent rebias) against numpy's conversion: bit-exact wherever it takes the value
    (including the rounding overflow to infinity just below 2^128), and it takes every
    input in [2^-126, 2^128); the rest goes to the FP64 definition."""
    u, _ = inputs(14, "f32")
    r = np.random.default_rng(15)
    # ties at bit 29, values around FP32's largest and smallest normal numbers
    tie = (np.uint64(1023 + r.integers(-100, 100, 3000)) << np.uint64(52)) | \
          (r.integers(0, 2 ** 23, 3000).astype(np.uint64) << np.uint64(29)) | np.uint64(1 << 28)
    big = np.ldexp(1.0 + r.random(2000) * 2.0 ** -20, 127) * (1.0 + 2.0 ** -23 * r.random(2000))
    big = np.concatenate([big, [float.fromhex("0x1.fffffefp127"), float.fromhex("0x1.ffffffp127"),
                                float.fromhex("0x1.fffffe8p127")]])
    small = np.ldexp(1.0 + r.random(2000), -126 + r.integers(-2, 3, 2000))
    u = np.concatenate([u, tie, big.view(np.uint64), small.view(np.uint64), (-small).view(np.uint64)])
    ok, t = run(harness, "f32fast", u, np.zeros(len(u), dtype=np.int64))
    x = u.view(np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        y = x.astype(np.float32)
    with np.errstate(invalid="ignore"):
        normal_in = np.isfinite(x) & (np.abs(x) >= 2.0 ** -126) & (np.abs(x) < 2.0 ** 128)
    assert np.all(ok[normal_in]), np.flatnonzero(normal_in & ~ok)[:10]
    assert np.array_equal(t[ok, 0], y[ok].view(np.uint32)), np.flatnonzero(t[ok, 0] != y[ok].view(np.uint32))[:10]
    assert np.any(ok & np.isinf(y)) and ok.sum() > 10000
