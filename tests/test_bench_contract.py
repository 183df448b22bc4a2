"""The reference arm of bench.py (the CPU oracle on bounded samples) keeps the JSON-line contract
on a small workload: one line on rank 0, no output on other ranks, and the keys the line must
carry (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nside", "32", "--lmax", "64",
           "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)


def test_reference_arm_prints_one_contract_line():
    r = run_reference()
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "maps/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    # ms_per_step is the measured wall time of one sample step; the value is extrapolated from it
    assert d["ms_per_step"] > 0
    assert "workload" in d["config"] and "Nside=32" in d["config"]["workload"]
    sys.path.insert(0, ROOT)
    import bench
    a = bench.argparse.Namespace(nside=32, lmax=64, maps=16)
    assert d["config"] == bench.workload_config(a)   # the same config object our arm prints
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["extrapolated"] is True and "extrapolated" in cb["sample"] and cb["cpu_model"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks():
    r = run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
