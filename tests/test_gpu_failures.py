"""Failure paths on the GPU, in forms that fault nothing.

* A bounded device wait that runs out: the FGMRES Arnoldi step's grid sync starts with
  an arrival count the host preset past its completion value (opts.expire_sync), so no
  block completes it; every block gives up after opts.wait_limit_us, records the expired
  wait in the handle's error word and returns.  The call reports LSQ_E_TIMEOUT and the
  next solve on the same handle succeeds.
* A NaN or an infinity placed in A or b on the host: the column-max pass records it and
  the call reports LSQ_E_NONFINITE (Sec. 1: the problem needs finite data).
"""
import time

import numpy as np
import pytest
import torch

from conftest import dev
from lsq_synth import paper_problem
from oracle import exact

pytestmark = pytest.mark.gpu

TIMEOUT, NONFINITE = -6, -4


def zeros(k):
    return torch.zeros(k, dtype=torch.float64, device="cuda")


def _solve_ok(lsq, handle, P):
    m, n = P.A.shape
    x, r = zeros(n), zeros(m)
    st, info = lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, 4 * n, "bf16", "f32", "f32", "f64", 1e-6, 0,
                            None, x, r)
    xstar, rstar = exact.reference_solution(P.A, P.b)
    ex, er = exact.forward_errors(x.cpu().numpy(), r.cpu().numpy(), xstar, rstar)
    assert st == 0 and ex <= 4 * 2.0 ** -24 and er <= 4 * 2.0 ** -24, (st, ex, er)


@pytest.mark.parametrize("arnoldi", [1, 2, 3])
def test_expired_wait_reports_timeout_and_handle_recovers(lsq, handle, arnoldi):
    """Classical (1) and modified (2: shared-memory work vector, 3: global) Arnoldi steps."""
    P = paper_problem(1e2, seed=5)
    m, n = P.A.shape
    x, r = zeros(n), zeros(m)
    t0 = time.time()
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_lsir(handle, dev(P.A), dev(P.b), m, n, 4 * n, "bf16", "f32", "f32", "f64", 1e-6, 0,
                     {"expire_sync": 1, "wait_limit_us": 20000, "arnoldi": arnoldi}, x, r)
    assert e.value.status == TIMEOUT
    assert time.time() - t0 < 30.0          # one expired 20 ms wait, the rest of the batch skipped
    _solve_ok(lsq, handle, P)               # same handle, no leftover error or barrier state


@pytest.mark.parametrize("where", ["A_nan", "A_inf", "b_nan", "b_ninf"])
def test_nonfinite_input_reports_nonfinite(lsq, handle, where):
    P = paper_problem(1e2, seed=6)
    m, n = P.A.shape
    A, b = P.A.copy(), P.b.copy()
    val = {"A_nan": np.nan, "A_inf": np.inf, "b_nan": np.nan, "b_ninf": -np.inf}[where]
    if where.startswith("A"):
        A[m // 3, n // 2] = val
    else:
        b[m - 1] = val
    x, r = zeros(n), zeros(m)
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_lsir(handle, dev(A), dev(b), m, n, 4 * n, "bf16", "f32", "f32", "f64", 1e-6, 0, None, x, r)
    assert e.value.status == NONFINITE
    Y = zeros(4 * n * (n + 1))
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_sketch(handle, dev(A), dev(b), m, n, 4 * n, "bf16", "f32", "f32", "f64", 1e-6, 0, None, Y)
    assert e.value.status == NONFINITE
    _solve_ok(lsq, handle, P)
