"""The stored oracle iteration counts (oracle/workload_counts.py: the oracle's full solve of
the m = 1e5, n = 500, kappa = 1e6 configuration) are for bench.py's secondary workload,
and the iteration counts the reference leg scales to are plausible for its main one."""
import bench
from oracle import workload_counts


def test_stored_oracle_counts_are_for_the_bench_workload():
    c = workload_counts.load()
    for k, v in c["workload"].items():
        assert bench.WL2[k] == v, k
    assert c["converged"]
    assert 1 <= c["lsqr_its"] <= 2 * bench.WL2["n"]
    assert c["ir_its"] == len(c["fgmres_its"]) and c["fgmres_total"] == sum(c["fgmres_its"])


def test_reference_leg_counts_are_within_the_caps():
    it = bench.GPU_ITERS
    assert 1 <= it["lsqr"] <= 2 * bench.WL["n"] and 1 <= it["fgmres"] <= 30 * 50
