"""The in-kernel sketch matrix fl_s(G) equals the oracle's definition bit for bit."""
import numpy as np
import pytest
import torch

from oracle import rng

pytestmark = pytest.mark.gpu

CASES = [(64, 0, 4096, 0), (33, 5, 1001, 12345), (8, 2 ** 32 - 6, 64, 2 ** 40 + 3),
         (5, 2 ** 34 + 1, 17, 7), (1, 3, 1, 99)]


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3", "bf16x3", "f32", "f64"])
def test_omega_bit_exact(lsq, handle, fmt):
    for s, j0, cols, seed in CASES:
        out = torch.full((s * cols,), float("nan"), dtype=torch.float64, device="cuda")
        lsq.lsq_omega(handle, s, j0, cols, fmt, seed, out)
        got = out.cpu().numpy().reshape(s, cols)
        ref = rng.sketch_operand(s, j0, j0 + cols, seed, fmt)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (fmt, s, j0, cols, seed)


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3"])
def test_omega_bit_exact_large_sample(lsq, handle, fmt):
    """4M entries: the FP32 evaluation with the FP64 fallback never rounds differently."""
    s, cols = 128, 32768
    out = torch.empty((s * cols,), dtype=torch.float64, device="cuda")
    lsq.lsq_omega(handle, s, 1 << 20, cols, fmt, 2024, out)
    got = out.cpu().numpy().reshape(s, cols)
    ref = rng.sketch_operand(s, 1 << 20, (1 << 20) + cols, 2024, fmt)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
