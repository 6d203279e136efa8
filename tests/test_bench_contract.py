"""The benchmark's reference arm (the CPU oracle timed on a bounded sample of the 24^4
workload) runs without a GPU: its JSON line carries the keys and values the benchmark
contract asks for, and under a multi-rank launch only rank 0 works and prints."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)


def test_reference_arm_line():
    p = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "dtype", "data", "scaling"):
        assert isinstance(d[key], str) and d[key]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_records_cpu_model_and_threads():
    p = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0", "OMP_NUM_THREADS": "3"})
    assert p.returncode == 0, p.stderr[-2000:]
    d = json.loads([ln for ln in p.stdout.splitlines() if ln.startswith("{")][0])
    assert d["cpu_baseline"]["cores"] == 3
    assert d["cpu_baseline"]["cpu_model"]


def test_roofline_fractions_recompute_from_the_line():
    """The roofline block carries every input of its fractions: algorithmic bytes per
    launch (updates per launch x bytes per update) over the average launch time, against
    the HBM, L2 and FMA peaks it names."""
    sys.path.insert(0, ROOT)
    import bench

    peaks = {"hbm_gbs": 6789.0, "l2_read_gbs": 18000.0, "fp64_fma_tflops": 1.2, "fp32_fma_tflops": 70.0}
    for prec, bpu in (("fp64", 72), ("fp32", 36)):
        r = bench.roofline_block(prec, 140.0, peaks)
        assert r["bytes_per_update"] == bpu
        achieved = r["updates_per_launch"] * bpu / (r["avg_launch_us"] * 1e-6) / 1e9
        assert abs(achieved / r["achieved"] - 1) < 1e-12
        assert abs(r["frac"] - achieved / peaks["hbm_gbs"]) < 1e-12
        assert abs(r["l2"]["frac"] - achieved / peaks["l2_read_gbs"]) < 1e-12
        assert abs(r["avg_launch_us"] * r["launches_per_step"] / 1e3 - 140.0) < 1e-9
        alu = r["updates_per_launch"] * r["alu"]["flop_per_update"] / (r["avg_launch_us"] * 1e-6) / 1e12
        assert abs(r["alu"]["frac"] - alu / r["alu"]["peak"]) < 1e-12
