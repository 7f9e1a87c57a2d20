"""Iteration counts of the oracle's full solve of the m = 1e5, n = 500 workload.

Test infrastructure only (see ``oracle/__init__.py``).  The reference leg of
``bench.py`` times the oracle on a row sample of this workload and scales the
per-iteration times to the number of LSQR and FGMRES iterations the oracle
itself takes to solve it; running the full oracle once per bench step would
take minutes.  ``python -m oracle.workload_counts`` reruns Algorithm 1 and
Algorithm 2 here (three-term BF16 sketch, FP32 QR, LSQR and FGMRES products,
FP64 residuals, the computable stop rule and the Sec. 5 escalation) and
rewrites ``workload_counts.json``; it calls only this package and the seeded
input generator.
"""
import json
import os
import time

import numpy as np

from . import lsir, qr, rng, sketch

WORKLOAD = dict(m=100000, n=500, s=2000, kappa=1e6, rho=1e-3, data_seed=1, seed=0, u_s="bf16x3",
                tol=1e-6)
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_counts.json")


def run(wl=WORKLOAD):
    from lsq_synth import randsvd_problem
    t0 = time.perf_counter()
    P = randsvd_problem(wl["m"], wl["n"], wl["kappa"], rho=wl["rho"], seed=wl["data_seed"])
    Y = sketch.sketch(P.A, P.b, wl["s"], wl["seed"], wl["u_s"])
    R, c = qr.householder_qr(Y, wl["n"], dtype=np.float32)
    x, r, info = lsir.lsir(P.A, P.b, R, qr.sketch_and_solve(R, c), 2.0 ** -24, wl["tol"],
                           w_dtype=np.float32, ur="f64", us=rng.UNIT_ROUNDOFF[wl["u_s"]],
                           kappa=wl["kappa"])
    return dict(workload=wl, lsqr_its=int(info["lsqr"]["its"]), ir_its=int(info["its"]),
                fgmres_its=[int(k) for k in info["gmres_its"]], fgmres_total=int(info["gmres_total"]),
                escalated=bool(info["escalated"]), converged=bool(info["converged"]),
                seconds=round(time.perf_counter() - t0, 1))


def load():
    with open(PATH) as fh:
        return json.load(fh)


if __name__ == "__main__":
    out = run()
    with open(PATH, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out))
