"""bench.py's JSON line carries every key of the benchmark contract, with values that
follow from its own timings (GPU arm run on CPU against a stubbed device and library,
tests/bench_mock_run.py: every CUDA event reports 10 ms)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args, env=None):
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bench_mock_run.py"), *args],
                         capture_output=True, text=True, timeout=900, cwd=ROOT,
                         env=dict(os.environ, **(env or {})))
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout[-2000:]
    return json.loads(lines[0])


def test_gpu_arm_line_follows_the_contract():
    steps = 2
    d = _line("--steps", str(steps), "--warmup", "3")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == 3
    assert d["higher_is_better"] is False and d["unit"] == "ms" and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and "workload" in d["config"]
    # one N = 1 job: K solves in the timed region, each event pair 10 ms
    assert d["value"] == d["ms_per_step"] == 10.0 / steps
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel"):
        assert k in r, k
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-12 * r["frac"]
    # the roofline names the kernel with the largest device time per solve
    ks = d["kernels"]
    assert r["kernel"] == max(ks, key=lambda k: ks[k]["total_ms"])
    assert d["tts_roofline"]["frac"] > 0
    c = d["cpu_baseline"]
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in c, k
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1
    e = d["e2e"]
    m, n = d["config"]["m"], d["config"]["n"]
    assert e["unit"] == "ms" and e["value"] > 0
    assert e["h2d_bytes_per_step"] == 8 * m * n + 8 * m and e["d2h_bytes_per_step"] > 0
    assert e["path"].startswith("lsq_lsir_host")       # host buffers through the C ABI
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    assert d["gpu_launches"] > 0


def test_e2e_failure_is_reported_not_fatal():
    d = _line("--steps", "1", "--warmup", "3", env={"BENCH_MOCK_HOST_CALL_FAILS": "1"})
    assert d["e2e"]["value"] is None and d["e2e"]["error"].startswith("RuntimeError")
    assert d["value"] == 10.0
