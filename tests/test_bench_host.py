"""The benchmark's host side on the CPU: the reference arm (the oracle timed on
the host cores) prints one JSON line with the contract's keys on rank 0 and
nothing on the other ranks; the roofline entry follows from its inputs."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    import bench

    lines = _run({"WORLD_SIZE": "1", "RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pts/s"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    # the value is the sample's targets over its measured wall time
    assert d["value"] > 0 and math.isclose(d["value"] * d["ms_per_step"] / 1e3, d["config"]["step_points"],
                                           rel_tol=1e-9)
    assert d["config"]["workload"] == bench.config(1)["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    assert _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []


def test_roofline_entry():
    import bench

    r = bench.roofline_entry(2.0e7, 87680, 78.5, "k", "note", traffic=None)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(2.0e7 * 87680 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 78.5)
