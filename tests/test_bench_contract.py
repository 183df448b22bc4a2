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


def test_ring_stage_figures_arithmetic():
    """The ring-stage figures of the bench line, on a hand-checked case: two rings of 4 and 8 pixels,
    mmax 3, 2 maps, 10 ms per call over 2 calls."""
    sys.path.insert(0, ROOT)
    import bench
    stages = {"ring_synth": (20.0, 2), "ring_anal": (40.0, 2), "legendre_synth": (99.0, 2)}
    seen = []

    def lookup(k):
        seen.append(k)
        return 8.0e6 if k == "ring_synth_kernel" else None

    r = bench.ring_stage_figures(stages, 2, 2, 2, 3, 12, [4, 8], 1000.0, 2.0, True, lookup)
    # Delta 2 maps x 2 rings x 4 m x 16 B = 256, maps 2 x 12 x 8 B = 192, phase table 2 x 4 x 16 B = 128
    alg = 256 + 192 + 128
    s = r["ring_synth"]
    assert s["algorithmic_bytes"] == alg and abs(s["ms_per_call"] - 10.0) < 1e-12
    assert abs(s["achieved_gbs"] - alg / 0.010 / 1e9) < 1e-15
    assert abs(s["hbm_frac"] - s["achieved_gbs"] / 1000.0) < 1e-18
    # 2.5 (4 log2 4 + 8 log2 8) = 2.5 (8 + 24) = 80 flops per map, 2 maps per call
    assert abs(s["fft_tflops_nominal"] - 160.0 / 0.010 / 1e12) < 1e-24
    assert abs(s["fp64_frac"] - s["fft_tflops_nominal"] / 2.0) < 1e-24
    assert s["traffic"] == 8.0e6 and abs(s["traffic_over_algorithmic"] - 8.0e6 / alg) < 1e-9
    a = r["ring_anal"]
    assert abs(a["ms_per_call"] - 20.0) < 1e-12 and a["traffic"] is None and a["traffic_over_algorithmic"] is None
    assert seen == ["ring_synth_kernel", "ring_anal_kernel"]
    assert "double-float" in r["note"]
    # the plain form: no traffic entries, FP64 wording; a stage with no launch is left out
    p = bench.ring_stage_figures({"ring_synth": (5.0, 1), "ring_anal": (0.0, 0)}, 1, 1, 2, 3, 12, [4, 8], 1000.0, 2.0)
    assert "traffic" not in p["ring_synth"] and "ring_anal" not in p and "FP64" in p["note"]
