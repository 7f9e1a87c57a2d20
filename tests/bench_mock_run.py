"""Runs bench.py's GPU arm on CPU with the device and the library stubbed out.

Test helper (not collected): ``python tests/bench_mock_run.py [bench args]``.
torch.cuda is replaced by no-op stand-ins (events report 10 ms), tensors stay
on the CPU, and the library returns fixed results, so that the bench's host
logic -- timing arithmetic, roofline, end-to-end leg, oracle legs and the JSON
line -- runs end to end on a small workload.
"""
import functools
import os
import sys
import types

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

EVENT_MS = 10.0

torch.cuda.is_available = lambda: True
torch.cuda.set_device = lambda *a: None
torch.cuda.synchronize = lambda *a: None


class _Stream:
    cuda_stream = 0


class _Event:
    def __init__(self, **kw):
        pass

    def record(self, *a):
        pass

    def elapsed_time(self, other):
        return EVENT_MS


torch.cuda.current_stream = lambda *a: _Stream()
torch.cuda.Event = _Event
torch.Tensor.cuda = lambda self, *a, **k: self
torch.Tensor.pin_memory = lambda self, *a, **k: self


def _cpu(f):
    @functools.wraps(f)
    def g(*a, **k):
        k.pop("device", None)
        k.pop("pin_memory", None)
        return f(*a, **k)
    return g


for _name in ("zeros", "empty", "full", "tensor"):
    setattr(torch, _name, _cpu(getattr(torch, _name)))

import paper_2410_06319_gb300._lib as real   # noqa: E402  (structs only; the library is not called)

fake = types.ModuleType("paper_2410_06319_gb300")
fake.KERNELS = real.KERNELS


class _Handle:
    def __init__(self, *a):
        pass

    def close(self):
        pass


def _lsir(h, A, b, m, n, s, *rest):
    info = real.Info()
    info.lsqr_its, info.ir_its, info.gmres_its_total, info.ir_converged = 7, 2, 80, 1
    info.gmres_its[0], info.gmres_its[1] = 40, 40
    for k in range(6):
        info.kern_ms[k] = 1.0
        info.kern_launches[k] = 10
    info.gpu_launches = 123
    return 0, info


def _lsir_host(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, x, r, info=None):
    if os.environ.get("BENCH_MOCK_HOST_CALL_FAILS"):
        raise RuntimeError("host call unavailable")
    x.zero_()                      # the stubbed device solve leaves x = 0, r = 0 as well
    if r is not None:
        r.zero_()
    return _lsir(h, A, b, m, n, s)


def _lsqr(h, A, b, m, n, s, *rest):
    info = real.Info()
    info.lsqr_its = 30
    return 0, info


def _ok(*a, **k):
    return 0


class _DeviceRandsvd:
    """The device generator on the CPU (same construction, small sizes)."""

    def __init__(self, m, n, seed=0, device=None):
        from lsq_synth import randsvd_problem
        self.m, self.n, self.seed = m, n, seed
        P = randsvd_problem(m, n, 1.0, rho=0.0, seed=seed)
        self.x_true = torch.from_numpy(P.x_true)

    def problem(self, kappa, rho):
        from lsq_synth import randsvd_problem
        P = randsvd_problem(self.m, self.n, kappa, rho=rho, seed=self.seed)
        self.x_true = torch.from_numpy(P.x_true)
        A = torch.from_numpy(P.A)
        return A, torch.from_numpy(P.b), torch.from_numpy(P.b - P.A @ P.x_true)

    def release(self):
        pass


def _batched(h, probs, *rest, **kw):
    infos = []
    for _ in probs:
        info = real.Info()
        info.ir_converged = 1
        infos.append(info)
    return 0, [0] * len(probs), infos


fake.Handle = _Handle
fake.lsq_lsir, fake.lsq_lsqr, fake.lsq_lsir_batched = _lsir, _lsqr, _batched
fake.lsq_lsir_host = _lsir_host
fake.lsq_sketch, fake.lsq_qr_r = _ok, _ok
fake.lsq_probe_fma_rate = lambda *a, **k: 5.0e11
sys.modules["paper_2410_06319_gb300"] = fake
import lsq_synth.device   # noqa: E402
lsq_synth.device.DeviceRandsvd = _DeviceRandsvd
torch.cuda.empty_cache = lambda *a: None

import bench   # noqa: E402

bench.WL.update(m=3000, n=60, s=240)
bench.WL2.update(m=2000, n=40, s=160)
bench.BATCH.update(count=2, m_range=(500, 600), n_range=(8, 10))
sys.argv = ["bench.py"] + sys.argv[1:]
bench.main()
