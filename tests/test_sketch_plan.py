"""The tensor-core sketch planner (host logic) against the limits its kernel relies on,
for every legal shape class: n up to 1024, s up to 16384, m up to 2^36.

The planner runs in the built library (no GPU needed).  Limits checked: the UMMA N
range (16..256, multiples of 16, M = 128), TMEM columns (a power of two, 32..512),
the TMA box (at most 256 rows; K step a multiple of 16 bytes), shared memory
(227 KB per CTA), grid dimensions, every column and every row of A covered exactly
once, and the 16-bit sketch-row field of the deferred-correction records.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06319_gb300", "csrc")
LIBDIR = os.path.join(ROOT, "paper_2410_06319_gb300", "_lib")
HARNESS = os.path.join(ROOT, "tests", "native", "plan_harness.cpp")
CUDA_INC = "/usr/local/cuda/include"

F16, BF16, E4M3, BF16X3 = 2, 3, 4, 5          # lsq_prec / kernel format codes
SMEM_MAX = 232448                              # 227 KB opt-in shared memory per CTA
Q_MAX = 256                                    # queued FP64 fallbacks per stage (exact mode)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    from test_lib_abi import load_builder
    load_builder().build()
    exe = str(tmp_path_factory.mktemp("plan") / "plan_harness")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                    HARNESS, "-L", LIBDIR, "-llsq", "-Wl,-rpath," + LIBDIR, "-o", exe], check=True)
    return exe


def shapes():
    ns = [1, 2, 15, 16, 17, 63, 127, 128, 254, 255, 256, 257, 300, 383, 500, 510, 511, 512, 513, 600,
          767, 1000, 1023, 1024]
    out = []
    for fmt in (F16, BF16, E4M3, BF16X3):
        for n in ns:
            for s in sorted({n, 2 * n + 1, 4 * n, min(16384, 16 * n), 16384}):
                if s < n:
                    continue
                for m in sorted({s, 4097, 100_000, 1_000_000, 4_000_000, 2 ** 31 + 5, 2 ** 36}):
                    if m < s:
                        continue
                    for sms in (152, 148, 1):
                        out.append((fmt, s, m, n + 1, sms))
    return out


def test_plans_respect_the_kernel_limits(harness):
    cases = shapes()
    text = "\n".join(" ".join(map(str, c)) for c in cases) + "\n"
    res = subprocess.run([harness], input=text, capture_output=True, text=True, check=True)
    lines = res.stdout.strip().splitlines()
    assert len(lines) == len(cases)
    for (fmt, s, m, ncols, sms), line in zip(cases, lines):
        f = [int(v) for v in line.split()]
        assert f[0] == 1, (fmt, s, m, ncols, sms)         # every legal shape has a plan
        _, bn, nsub, ngroups, mtiles, splits, kchunk, s_pad, stages, nt, rowb, smem, cap, lists = f
        ctx = (fmt, s, m, ncols, sms, f)
        eb = 1 if fmt == E4M3 else 2
        chunk = bn // nsub
        # MMA shape (M = 128): N a multiple of 16 in [16, 256]; columns covered
        assert nsub in (1, 2) and bn % nsub == 0 and chunk % 16 == 0 and 16 <= chunk <= 256, ctx
        assert ngroups * bn >= ncols and (ngroups - 1) * bn < ncols, ctx
        tmem = 32
        while tmem < bn:
            tmem *= 2
        assert tmem <= 512, ctx
        # operand planes and swizzle: 3 BF16 planes use 64-byte rows, one plane 128-byte rows
        assert nt == (3 if fmt == BF16X3 else 1) and rowb == (64 if nt == 3 else 128), ctx
        bk = rowb // eb                                   # K elements per stage
        assert (bk * eb) % 16 == 0 and chunk <= 256, ctx  # TMA: 16-byte x steps, box rows <= 256
        # shared memory: stage ring + barriers + fallback queues
        stage = 128 * rowb + nt * bn * rowb
        assert stages in (2, 4), ctx
        assert smem == 1024 + stages * stage + 512 + stages * Q_MAX * 12 and smem <= SMEM_MAX, ctx
        # K split: whole K steps, every row of A in exactly one split, no empty split
        assert kchunk % bk == 0 and splits * kchunk >= m and (splits - 1) * kchunk < m, ctx
        assert mtiles == (s + 127) // 128 and s_pad >= s, ctx
        assert splits <= 65535 and ngroups <= 65535 and mtiles < 2 ** 31, ctx
        # deferred records pack (data row << 16 | sketch row): sketch rows below 2^16
        assert mtiles * 128 <= 2 ** 16 and m < 2 ** 48, ctx
        assert 0 < cap < 2 ** 32 and lists == mtiles * ngroups * splits * 16, ctx


def test_configurations_keep_the_deferred_correction(harness):
    """The correction lists (records of 8 bytes) of the workloads run at full size stay
    below the 4 GiB past which the sketch switches to its exact in-pipeline mode."""
    cases = [(BF16X3, 2000, 100_000, 501), (BF16, 2000, 100_000, 501), (F16, 2000, 100_000, 501),
             (F16, 3000, 1_000_000, 1001), (E4M3, 3000, 1_000_000, 1001),
             (BF16, 4000, 4_000_000, 1001), (BF16X3, 4000, 4_000_000, 1001)]
    text = "\n".join(f"{f} {s} {m} {c} 152" for f, s, m, c in cases) + "\n"
    res = subprocess.run([harness], input=text, capture_output=True, text=True, check=True)
    for case, line in zip(cases, res.stdout.strip().splitlines()):
        f = [int(v) for v in line.split()]
        assert f[0] == 1 and f[12] * f[13] * 8 <= 4 << 30, (case, f[12] * f[13] * 8)
