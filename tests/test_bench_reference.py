"""The reference leg of bench.py scales the oracle's sampled per-iteration times to
the oracle's own iteration counts on the workload (stored by oracle/workload_counts.py):
those counts must be for the workload bench.py runs."""
import bench
from oracle import workload_counts


def test_stored_oracle_counts_are_for_the_bench_workload():
    c = workload_counts.load()
    for k, v in c["workload"].items():
        assert bench.WL[k] == v, k
    assert c["converged"]
    assert 1 <= c["lsqr_its"] <= 2 * bench.WL["n"]
    assert c["ir_its"] == len(c["fgmres_its"]) and c["fgmres_total"] == sum(c["fgmres_its"])
