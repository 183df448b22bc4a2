#!/usr/bin/env python
"""Benchmark: alm2map + map2alm round trips at lmax = mmax = 4096 on HEALPix
Nside = 2048 (50,331,648 pixels), a batch of maps per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode split|fp64]

One step = sht_alm2map of B maps followed by sht_map2alm of the result
(B = --maps, default 16), in the precision form by default (FP64
recurrence, tensor-core synthesis sum, double-float analysis sum).  `value`
is maps per second (round trips) over the whole job with inputs resident in
HBM; `e2e` is the same metric with the host->device copy of each step's a_lm
(pinned) and the device->host read of its result inside the timed region.
The same line carries the plain FP64 form measured in the same run (`plain`),
the precision form's error against the plain path and the oracle
(`accuracy`), a Poisson serving trace served by the continuous-batching
server against the plain one-at-a-time path (`serve`: maps/s at saturation,
p50/p99 latency at the offered rate) and the batched form (`batched`: 256
maps of mixed lmax and direction as one CUDA graph, FP64 and precision form).
For N > 1 (torchrun) every rank runs an independent replica of the workload;
the barrier-bracketed time is the max over ranks.  `--impl reference` times
the CPU oracle on this host's cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SM_MAX_MHZ = 2070  # GB300 maximum SM clock


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


MEASURED = _measured_peaks()
METRIC = "ℓmax=4096 alm2map+map2alm maps/s, served vs plain; p99 ms; % FP64/TC peak"
DATA = "synthetic: seeded complex Gaussian a_lm with C_l = 1/(l(l+1)+1), a_l0 real (CMB-like)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nside", type=int, default=2048)
    ap.add_argument("--lmax", type=int, default=4096)
    ap.add_argument("--maps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", default="split", choices=["split", "fp64"],
                    help="split: precision form, tensor-core synthesis and analysis (<= 1e-9); fp64: plain")
    ap.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain FP64 comparison")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests in the serving trace (0: no serving leg)")
    ap.add_argument("--batch-maps", type=int, default=256, help="maps in the batched-form leg (0: no batched leg)")
    ap.add_argument("--no-c2", dest="c2", action="store_false",
                    help="skip the plain FP64 lmax = 2048 leg (HEALPix 1024 and the Gauss-Legendre round trip)")
    ap.add_argument("--prec-anal", default="tc", choices=["df", "tc"],
                    help="precision-form analysis kernel: tensor cores (default) or double-float")
    return ap.parse_args()


MODES = {"split": "precision form: FP64 recurrence, tensor-core (tcgen05, split-bf16, 7 digits) synthesis "
                  "sum, %s analysis sum",
         "fp64": "plain FP64"}


def mode_desc(a, mode=None):
    mode = mode or a.mode
    if mode != "split":
        return MODES[mode]
    return MODES[mode] % ("tensor-core (split-bf16)" if a.prec_anal == "tc" else "double-float (FP32 pipe)")


def workload_name(a):
    return ("alm2map then map2alm round trip, HEALPix Nside=%d (%d px, %d rings), lmax=mmax=%d, "
            "%d maps per step" % (a.nside, 12 * a.nside ** 2, 4 * a.nside - 1, a.lmax, a.maps))


# ---------------------------------------------------------------- clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle on bounded samples

def oracle_sample(nside, lmax, nrings_sample, nm_sample, offset=0, alm=None, smap=None):
    """Time the oracle on `nrings_sample` rings of alm2map and `nm_sample` values of m of
    map2alm (either may be 0); return (seconds per ring, seconds per m, description, sample)
    where sample holds the rings, the values of m and the oracle's outputs there (for accuracy
    checks).  The oracle's parallel loops run over the selected rings and values of m, so a
    sample of at least as many items as host threads keeps every core busy."""
    import numpy as np

    import oracle
    from oracle import geometry
    from paper_1106_0159_gb300 import inputs

    geom = geometry.healpix(nside)
    R = len(geom[0])
    rings = [int((offset + (k + 0.5) * R / max(nrings_sample, 1))) % R for k in range(nrings_sample)]
    ms = [int((offset * 7 + (k + 0.5) * (lmax + 1) / max(nm_sample, 1))) % (lmax + 1) for k in range(nm_sample)]
    ring_vals, alm_vals, tr, tm = None, None, 0.0, 0.0
    if rings:
        a = inputs.gaussian_alm(lmax, lmax, seed=100)[0] if alm is None else alm
        t0 = time.perf_counter()
        ring_vals = oracle.alm2map_rings(geom, a, lmax, lmax, rings)
        tr = time.perf_counter() - t0
    if ms:
        s = inputs.white_map(int(np.sum(geom[0])), seed=101)[0] if smap is None else smap
        t0 = time.perf_counter()
        alm_vals = oracle.map2alm_ms(geom, s, lmax, ms)
        tm = time.perf_counter() - t0
    desc = ("oracle alm2map on %d of %d rings (%.1f s wall) + map2alm on %d of %d values of m (%.1f s wall)"
            % (len(rings), R, tr, len(ms), lmax + 1, tm))
    per_ring = tr / len(rings) if rings else None
    per_m = tm / len(ms) if ms else None
    return per_ring, per_m, desc, {"rings": rings, "ring_vals": ring_vals, "ms": ms, "alm_vals": alm_vals}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline lines."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def workload_config(a):
    """The `config` object both arms print: the workload, not the arm's arithmetic."""
    return {"workload": workload_name(a), "grid": "HEALPix", "nside": a.nside, "lmax": a.lmax,
            "mmax": a.lmax, "maps_per_step": a.maps, "directions": "alm2map then map2alm",
            "accuracy": "<= 1e-9 of the RMS vs the oracle (precision form); <= 1e-11 (FP64)",
            "l2": "inputs larger than L2 (a_lm %.2f GB, maps %.2f GB per step)"
                  % (a.maps * (a.lmax + 1) * (a.lmax + 2) / 2 * 16 / 1e9, a.maps * 12 * a.nside ** 2 * 8 / 1e9)}


def reference_arm(a, rank, world):
    """The oracle on this host's cores.  Timed step k samples 16 rings of alm2map (k even) or 16
    values of m of map2alm (k odd), rotating over the sphere; the value is one full round trip
    per map extrapolated from the mean seconds per ring and per m over all timed steps (a
    measured sample, scaled, not a full run).  Warm-up steps sample one value of m."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nthr = host_threads()
    k_items = 16
    for i in range(a.warmup):
        oracle_sample(a.nside, a.lmax, 0, 1, offset=i)
    ring_t, m_t, step_s = [], [], []
    for i in range(a.steps):
        t0 = time.perf_counter()
        pr, pm, _, _ = oracle_sample(a.nside, a.lmax, k_items if i % 2 == 0 else 0, 0 if i % 2 == 0 else k_items,
                                     offset=i)
        step_s.append(time.perf_counter() - t0)
        if pr is not None:
            ring_t.append(pr)
        if pm is not None:
            m_t.append(pm)
    if not m_t:  # a single timed step: sample m once more so that both halves are measured
        m_t.append(oracle_sample(a.nside, a.lmax, 0, k_items, offset=a.steps)[1])
    R = 4 * a.nside - 1
    per_map_s = statistics.mean(ring_t) * R + statistics.mean(m_t) * (a.lmax + 1)
    value = 1.0 / per_map_s
    sample = ("extrapolated, not a full run: %d timed steps, each 16 rings of alm2map or 16 values of m of "
              "map2alm (alternating, rotating offsets), %.2f s per ring and %.3f s per m (wall, %d threads), "
              "scaled to %d rings + %d values of m = %.0f s per map round trip" %
              (a.steps, statistics.mean(ring_t), statistics.mean(m_t), nthr, R, a.lmax + 1, per_map_s))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "maps/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(step_s) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "long double (80-bit x87 or binary128) CPU oracle", "data": DATA,
        "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": "maps/s", "cores": nthr, "kind": "oracle",
                         "cpu_model": cpu_model(), "extrapolated": True, "sample": sample},
        "e2e": {"value": value, "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "ms_per_step is the measured wall time of one sample step; value is extrapolated to full "
                "map round trips from the per-ring and per-m times",
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def traffic_from_profiles(kernel_key):
    """DRAM bytes per launch recorded by an ncu capture, if the kernel source is unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p)).get(kernel_key)
    except Exception:
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_1106_0159_gb300", "csrc", rec.get("source", ""))
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    if sha != rec.get("source_sha256_16"):
        return None
    return rec.get("bytes_per_launch")


def ring_stage_figures(stages, steps, nmaps, nrings, mmax, npix, nphi, hbm_peak_gbs, fp64_peak_tflops,
                       double_float=False, traffic_lookup=None):
    """Ring stages (eqs. Delta2map and almfftdef), one launch per call and direction, from the
    per-stage CUDA-event times {name: (ms over `steps` calls, launches)}.  Algorithmic bytes per
    call: Delta (nmaps x nrings x (mmax + 1) complex128, written or read) + maps (nmaps x npix
    float64, read or written) + the phase table once (nrings x (mmax + 1) x 16 B).  Nominal FFT
    work: 2.5 n log2 n flops per real ring of n pixels and map (a complex DFT of length n carries
    two rings at 5 n log2 n); Bluestein's extra work is not counted.  `double_float`: the DFTs ran in
    double-float arithmetic (FP32 pipe); `traffic_lookup(kernel)` gives the recorded DRAM bytes of a
    launch (the double-float DFTs at 16 maps), or None."""
    import numpy as np

    nphi = np.asarray(nphi, dtype=np.float64)
    fft_flops_map = float(2.5 * np.sum(nphi * np.log2(nphi)))
    alg = nmaps * (nrings * (mmax + 1) * 16 + npix * 8) + nrings * (mmax + 1) * 16
    out = {}
    for key in ("ring_synth", "ring_anal"):
        ms, n = stages.get(key, (0.0, 0))
        if not n:
            continue
        per_call_s = ms * 1e-3 / steps
        gbs = alg / per_call_s / 1e9
        tf = nmaps * fft_flops_map / per_call_s / 1e12
        r = {"ms_per_call": per_call_s * 1e3, "algorithmic_bytes": alg, "achieved_gbs": gbs,
             "hbm_peak_gbs": hbm_peak_gbs, "hbm_frac": gbs / hbm_peak_gbs, "fft_tflops_nominal": tf,
             "fp64_peak_tflops": fp64_peak_tflops, "fp64_frac": tf / fp64_peak_tflops}
        if traffic_lookup is not None:
            tr = traffic_lookup(key + "_kernel")
            r["traffic"] = tr
            r["traffic_over_algorithmic"] = (tr / alg) if tr else None
        out[key] = r
    out["note"] = ("nominal FFT flops (no Bluestein overhead) over the stage's CUDA-event time; %s" %
                   ("double-float arithmetic on the FP32 pipe: fp64_frac is the FP64-equivalent rate"
                    if double_float else "FP64 arithmetic"))
    return out


def ours_arm(a, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1106_0159_gb300 import inputs, sht

    from paper_1106_0159_gb300.replicas import Replicas, job_throughput

    torch.cuda.set_device(local_rank)
    rep = Replicas(device=torch.device("cuda", local_rank))
    barrier = rep.barrier

    sht.load()
    probe_tf = sht.fp64_fma_tflops()
    # FP64 pipe: 2 FMA per SM per cycle (ncu: FP32:FP64 = 64:1 on this part) at the maximum SM clock
    nsm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak_tf = 2 * 2 * nsm * SM_MAX_MHZ * 1e6 / 1e12
    geom = sht.healpix_geometry(a.nside)
    t0 = time.perf_counter()
    plan = sht.Plan(geom, a.lmax, a.lmax, grid=sht.GRID_HEALPIX)
    plan_s = time.perf_counter() - t0
    B, L = a.maps, a.lmax
    nalm, npix = plan.nalm, plan.npix
    host_alm = torch.from_numpy(inputs.gaussian_alm(L, L, seed=rep.seed(1000), nmaps=B)).pin_memory()
    alm = host_alm.cuda()
    mp = torch.empty((B, npix), dtype=torch.float64, device="cuda")
    alm_out = torch.empty((B, nalm), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.alm2map(alm, out=mp)
        plan.map2alm(mp, out=alm_out)

    plan.set_tuning(sht.TUNE_PREC_ANAL, 1 if a.prec_anal == "tc" else 0)

    def timed(mode, steps, warmup, sample_clocks):
        plan.set_mode(sht.MODE_SPLIT_BF16 if mode == "split" else sht.MODE_FP64)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        plan.set_stage_timing(True)
        plan.stage_times(reset=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        clocks = ClockSampler(local_rank) if sample_clocks else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        evs[0].record(stream)
        for i in range(steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        total = rep.max_over_ranks(evs[0].elapsed_time(evs[-1]), device="cuda")
        stages = plan.stage_times(reset=True)
        plan.set_stage_timing(False)
        return {"total_ms": total, "step_ms": step_ms, "stages": stages, "clocks": clk}

    S = sum(L - m + 1 for m in range(L + 1)) * plan.npairs  # (l, m, ring-pair) steps of one transform

    def fp64_roofline(run, steps):
        # dominant Legendre stage on the FP64 pipe: nominal 3 flops per step for each launch's
        # recurrence plus 4 flops per step per map for the accumulation
        legendre = {k: v for k, v in run["stages"].items() if k in ("legendre_synth", "legendre_anal")}
        dom = max(legendre, key=lambda k: legendre[k][0])
        dom_ms, dom_launches = legendre[dom]
        flops = S * (3.0 * dom_launches + 4.0 * B * steps)
        achieved = flops / (dom_ms * 1e-3) / 1e12
        key = "legendre_anal_kernel" if dom == "legendre_anal" else "legendre_synth_kernel"
        return {"bound": "alu", "pipe": "fp64", "kernel": key, "achieved": achieved, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": traffic_from_profiles(key),
                "peak_source": "derived: 2 FP64 FMA/clk/SM x %d SMs x %d MHz x 2 flop; in-run FMA probe %.3f "
                               "TF/s" % (nsm, SM_MAX_MHZ, probe_tf),
                "work": "7 flops per (l, m, ring-pair) step over the full triangle, per map (3 recurrence + 4 "
                        "accumulate); steps whose lambda is below 2^-224 are skipped, so frac can exceed 1",
                "time": "the Legendre stage (all its launches)",
                "live_share": live_share, "frac_of_executed": achieved / peak_tf * live_share}

    # live share of the (l, m, ring-pair) steps: the precision-form tables mark the first 32-l chunk
    # per (m, 128-slot block) above the dropping threshold; the plain kernels skip the same prefix
    # per warp, so the nominal fractions below count about 1 / live more work than is executed
    plan.set_mode(sht.MODE_SPLIT_BF16)
    live_steps, total_steps = plan.live_steps()
    live_share = live_steps / total_steps

    def split_roofline(run, steps):
        st = run["stages"]
        if plan.tuning(sht.TUNE_PREC_ANAL) == 0 and st["legendre_anal"][0] >= st["legendre_synth"][0]:
            # double-float analysis on the FP32 pipe: per (l, m, ring-pair, map) two real products
            # (1 FMUL + 3 FFMA = 7 flops each) and their double-float sums (TwoSum + 2 adds = 8 flops)
            ms = st["legendre_anal"][0]
            peak = 2 * 128 * nsm * SM_MAX_MHZ * 1e6 / 1e12
            achieved = 30.0 * S * B * steps / (ms * 1e-3) / 1e12
            return {"bound": "alu", "pipe": "fp32", "kernel": "legendre_anal_df_kernel", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic_from_profiles("legendre_anal_df_kernel"),
                    "peak_source": "derived: 128 FP32 FMA/clk/SM x %d SMs x %d MHz x 2 flop" % (nsm, SM_MAX_MHZ),
                    "work": "30 FP32 flops per (l, m, ring-pair, map): two double-float real products and sums",
                    "time": "analysis stage (includes the polar kernel and the block reduction)"}
        # the tensor-core kernels, each timed alone by its own CUDA events on the call's stream
        # (stage ids tc_synth_kernel / tc_anal_kernel: no polar kernel, no block reduction)
        ka_ms, ka_n = st["tc_anal_kernel"]
        ks_ms, ks_n = st["tc_synth_kernel"]
        anal = ka_ms >= ks_ms
        ms, nl = (ka_ms, ka_n) if anal else (ks_ms, ks_n)
        key = "tc_anal_kernel" if anal else "tc_synth_kernel"
        groups = -(-B // 16) * steps            # passes of the recurrence: one per group of <= 16 maps
        per_group_s = ms * 1e-3 / groups         # the analysis runs a group as about eight m-slab launches
        maps_per_group = min(B, 16)
        # binding pipe: the tensor cores.  Useful work = the 28 digit-pair slice-products, each the
        # whole contraction of 4 flops per (l, m, ring-pair) step and map (complex x real), over the
        # full triangle S
        tflops = 28 * 4.0 * maps_per_group * S / per_group_s / 1e12
        tpeak = MEASURED.get("bf16_tflops_sustained") or 1725.1
        # the FP64 recurrence beside it: 3 flops per step, once per group
        fflops = 3.0 * S / per_group_s / 1e12
        # algorithmic bytes per group: Delta read and a_lm written (analysis), a_lm read and
        # Delta written (synthesis)
        alg = maps_per_group * (plan.nrings * (L + 1) + nalm) * 16
        traffic = traffic_from_profiles(key)
        return {"bound": "tensor", "kernel": key, "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s",
                "frac": tflops / tpeak, "traffic": traffic,
                "peak_source": "measured bf16 GEMM, sustained (MEASURED_PEAKS.json bf16_tflops_sustained): the "
                               "kernel is timed inside a long step",
                "work": "28 bf16 digit-pair products x 4 flops per (l, m, ring-pair) step and map, nominal full "
                        "triangle S = %d steps, %d maps per group: %.3e flops per group" %
                        (S, maps_per_group, 28 * 4.0 * maps_per_group * S),
                "time": "the kernel's own launches (CUDA events around each launch on the call's stream): "
                        "%.2f ms per group of %d maps, %d launches in %d groups" %
                        (per_group_s * 1e3, maps_per_group, nl, groups),
                "live_share": live_share,
                "frac_of_executed": tflops / tpeak / live_share,
                "fp64": {"achieved": fflops, "peak": peak_tf, "unit": "TFLOP/s", "frac": fflops / peak_tf,
                         "work": "3 FP64 flops per (l, m, ring-pair) step of the recurrence, once per launch",
                         "peak_source": "derived: 2 FP64 FMA/clk/SM x %d SMs x %d MHz x 2 flop; in-run FMA probe "
                                        "%.3f TF/s" % (nsm, SM_MAX_MHZ, probe_tf)},
                "algorithmic_bytes": alg,
                "traffic_over_algorithmic": (traffic / alg) if traffic else None}

    hbm_peak = MEASURED.get("hbm_gbs") or 6800.0

    def ring_stages(run, steps, double_float):
        return ring_stage_figures(run["stages"], steps, B, plan.nrings, L, npix, geom[0], hbm_peak, peak_tf,
                                  double_float, traffic_from_profiles if double_float and B == 16 else None)

    head = timed(a.mode, a.steps, a.warmup, True)
    total_ms, step_ms, stages, clk = head["total_ms"], head["step_ms"], head["stages"], head["clocks"]
    value = job_throughput(world, B * a.steps, total_ms)
    roofline = split_roofline(head, a.steps) if a.mode == "split" else fp64_roofline(head, a.steps)
    launches = sum(v[1] for v in stages.values())

    plain = None
    if a.mode == "split" and a.plain_steps > 0:
        pr = timed("fp64", a.plain_steps, 1, False)
        plain = {"value": job_throughput(world, B * a.plain_steps, pr["total_ms"]), "unit": "maps/s",
                 "ms_per_step": pr["total_ms"] / a.plain_steps, "steps": a.plain_steps, "warmup": 1,
                 "stages_ms_per_step": {k: v[0] / a.plain_steps for k, v in pr["stages"].items()},
                 "roofline": fp64_roofline(pr, a.plain_steps),
                 "ring_stages": ring_stages(pr, a.plain_steps, False)}
        plan.set_mode(sht.MODE_SPLIT_BF16)

    # end to end: pinned host a_lm -> device, round trip, result back to pinned host memory, every
    # step.  The copies run on a copy stream, double-buffered, so that step i + 1's upload and step
    # i's download overlap step i's transforms (a pipeline over a stream of batches).  The timed
    # region runs from the first upload to the last download.
    e2e = None
    if not a.no_e2e:
        host_out = torch.empty((B, nalm), dtype=torch.complex128).pin_memory()
        copy = torch.cuda.Stream()
        ins = [alm, torch.empty_like(alm)]
        outs = [alm_out, torch.empty_like(alm_out)]
        ev = torch.cuda.Event

        def run_pipeline(nsteps):
            up = [ev(), ev()]          # upload of buffer b done
            done = [ev(), ev()]        # transforms that read ins[b] / wrote outs[b] done
            down = [ev(), ev()]        # download of outs[b] done
            started = [False, False]
            t0, t1 = ev(enable_timing=True), ev(enable_timing=True)
            t0.record(copy)
            with torch.cuda.stream(copy):
                ins[0].copy_(host_alm, non_blocking=True)
            up[0].record(copy)
            for i in range(nsteps):
                b = i & 1
                if i + 1 < nsteps:  # next upload into the other buffer, once its last transforms finished
                    nb = b ^ 1
                    if started[nb]:
                        copy.wait_event(done[nb])
                    with torch.cuda.stream(copy):
                        ins[nb].copy_(host_alm, non_blocking=True)
                    up[nb].record(copy)
                stream.wait_event(up[b])
                if started[b]:
                    stream.wait_event(down[b])  # outs[b] was read back
                plan.alm2map(ins[b], out=mp)
                plan.map2alm(mp, out=outs[b])
                done[b].record(stream)
                started[b] = True
                copy.wait_event(done[b])
                with torch.cuda.stream(copy):
                    host_out.copy_(outs[b], non_blocking=True)
                down[b].record(copy)
            t1.record(copy)
            return t0, t1

        run_pipeline(2)
        torch.cuda.synchronize()
        barrier()
        t0, t1 = run_pipeline(a.steps)
        torch.cuda.synchronize()
        barrier()
        ems = rep.max_over_ranks(t0.elapsed_time(t1), device="cuda")
        nbytes = B * nalm * 16
        e2e = {"value": job_throughput(world, B * a.steps, ems), "unit": "maps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "form": "uploads and downloads on a copy stream, double-buffered, overlapping the transforms"}

    # accuracy of the precision form: against the plain FP64 path on the whole timed batch, both
    # directions on the same inputs (max |x - x_plain| / RMS(x_plain), worst map)
    accuracy = None
    if a.mode == "split":
        def rel_maps(x, ref):
            d = (x - ref).abs().amax(dim=1)
            r = ref.abs().pow(2).mean(dim=1).sqrt()
            return float((d / r).max())

        plan.set_mode(sht.MODE_FP64)
        plan.alm2map(alm, out=mp)
        plan.map2alm(mp, out=alm_out)
        alm_plain = alm_out.clone()
        plan.set_mode(sht.MODE_SPLIT_BF16)
        map_split = torch.empty_like(mp)
        plan.alm2map(alm, out=map_split)
        plan.map2alm(mp, out=alm_out)          # analysis of the plain map: the same input both ways
        torch.cuda.synchronize()
        accuracy = {"split_vs_plain_fp64": {"alm2map": rel_maps(map_split, mp), "map2alm": rel_maps(alm_out, alm_plain),
                                            "maps": B, "measure": "max|x - x_plain| / RMS(x_plain), worst map"},
                    "bar": 1e-9}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        nthr = host_threads()
        a0 = host_alm[0].numpy()
        s0 = mp[0].cpu().numpy() if accuracy else None
        k_items = 16
        pr, pm, desc, smp = oracle_sample(a.nside, a.lmax, k_items, k_items, alm=a0, smap=s0)
        per_map_s = pr * plan.nrings + pm * (L + 1)
        cpu = {"value": 1.0 / per_map_s, "unit": "maps/s", "cores": nthr, "kind": "oracle",
               "cpu_model": cpu_model(), "extrapolated": True,
               "sample": "extrapolated, not a full run: " + desc + ", %.2f s per ring and %.3f s per m, scaled to "
                         "%d rings + %d values of m = %.0f s per map round trip" %
                         (pr, pm, plan.nrings, L + 1, per_map_s)}
        if accuracy:
            # the same oracle outputs checked against map 0 of the batch (rings and m of the sample)
            ofs = np.concatenate([[0], np.cumsum(np.asarray(geom[0], dtype=np.int64))])
            pix = np.concatenate([np.arange(ofs[r], ofs[r + 1]) for r in smp["rings"]])
            ref = smp["ring_vals"]
            rms = np.sqrt(np.mean(ref ** 2))
            got_s = map_split[0].cpu().numpy()[pix]
            got_p = mp[0].cpu().numpy()[pix]
            idx = np.concatenate([[sht.alm_index(L, l, m) for l in range(m, L + 1)] for m in smp["ms"]])
            aref = np.concatenate(smp["alm_vals"])
            arms = np.sqrt(np.mean(np.abs(aref) ** 2))
            accuracy["vs_oracle_sampled"] = {
                "alm2map_split": float(np.max(np.abs(got_s - ref)) / rms),
                "alm2map_plain": float(np.max(np.abs(got_p - ref)) / rms),
                "map2alm_split": float(np.max(np.abs(alm_out[0].cpu().numpy()[idx] - aref)) / arms),
                "map2alm_plain": float(np.max(np.abs(alm_plain[0].cpu().numpy()[idx] - aref)) / arms),
                "sample": "map 0: %d rings %s of alm2map; m = %s of map2alm (input: the plain map); "
                          "normalised by the RMS of the oracle's sampled values" % (len(smp["rings"]), smp["rings"],
                                                                                   smp["ms"])}

    if rank == 0:
        q = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "maps/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f64 recurrence; synthesis: bf16 digits (tcgen05, f32 accum, f64 combination); analysis: "
                      + ("bf16 digits (tcgen05)" if a.prec_anal == "tc" else "double-float (f32 pairs)"))
                     if a.mode == "split" else "f64",
            "data": DATA,
            "config": workload_config(a),
            "mode": mode_desc(a), "parallelism": "replicas" if world > 1 else "single GPU",
            "plan_create_s": plan_s,
            "latency_ms": {"p50": statistics.median(q), "p99": q[min(len(q) - 1, int(0.99 * len(q)))],
                           "per": "step (%d-map round trip)" % B},
            "roofline": roofline,
            "stages_ms_per_step": {k: v[0] / a.steps for k, v in stages.items()},
            "ring_stages": ring_stages(head, a.steps, a.mode == "split" and plan.tuning(sht.TUNE_PREC_RING) == 1),
            "plain": plain,
            "accuracy": accuracy,
            "serve": None,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
    del alm, mp, alm_out, host_alm
    if accuracy:
        del alm_plain, map_split
    plan.close()
    torch.cuda.empty_cache()
    serve_res = serve_leg(a, rep, local_rank) if a.serve_requests > 0 else None
    batch_res = batch_leg(a, rep, local_rank) if a.batch_maps > 0 else None
    c2_res = c2_leg(a, rep, local_rank, nsm, peak_tf) if a.c2 else None
    if rank == 0:
        line["serve"] = serve_res
        line["batched"] = batch_res
        line["c2_plain_fp64_lmax2048"] = c2_res
        if cpu is not None:
            cpu["o1_c1"] = o1_leg()
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


def _flush_l2(buf):
    buf.add_(1.0)  # a write larger than L2 between timed repetitions


def c2_leg(a, rep, local_rank, nsm, peak_tf):
    """Plain FP64 at lmax = mmax = 2048, one map per call: alm2map and map2alm on HEALPix Nside
    1024 (12.6 M pixels), each timed alone, and the Gauss-Legendre 2049 x 4097 round trip with
    its error (the quadrature is exact there, so map2alm(alm2map(a)) = a).  Each repetition is
    timed with its own CUDA events after an L2 flush (the inputs fit in L2 at this size)."""
    import numpy as np
    import torch

    from paper_1106_0159_gb300 import inputs, sht

    L, reps = 2048, 3
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            _flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    out = {}
    for name, geom, grid, inp in (("healpix1024", sht.healpix_geometry(1024), sht.GRID_HEALPIX, "gaussian"),
                                  ("gl2049x4097", sht.gauss_legendre_geometry(2049, 4097),
                                   sht.GRID_GAUSS_LEGENDRE, "uniform")):
        plan = sht.Plan(geom, L, L, grid=grid)
        if inp == "gaussian":
            ah = inputs.gaussian_alm(L, L, seed=rep.seed(2048), nmaps=1)
        else:
            ah = inputs.uniform_alm(L, L, seed=rep.seed(2049), nmaps=1)
        alm = torch.from_numpy(ah).cuda()
        mp = torch.empty((1, plan.npix), dtype=torch.float64, device="cuda")
        back = torch.empty((1, plan.nalm), dtype=torch.complex128, device="cuda")
        plan.alm2map(alm, out=mp)
        plan.set_stage_timing(True)
        plan.stage_times(reset=True)
        t_syn = timed(lambda: plan.alm2map(alm, out=mp))
        st_syn = plan.stage_times(reset=True)
        t_ana = timed(lambda: plan.map2alm(mp, out=back))
        st_ana = plan.stage_times(reset=True)
        plan.set_stage_timing(False)
        S = sum(L - m + 1 for m in range(L + 1)) * plan.npairs
        n = reps + 1

        def roof(ms_total):
            ach = 7.0 * S / (ms_total / n * 1e-3) / 1e12
            return {"achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf}

        r = {"npix": plan.npix, "nrings": plan.nrings, "alm2map_ms": t_syn, "map2alm_ms": t_ana,
             "round_trip_maps_per_s": 1e3 / (t_syn + t_ana),
             "stages_ms": {"alm2map": {k: v[0] / n for k, v in st_syn.items() if v[1]},
                           "map2alm": {k: v[0] / n for k, v in st_ana.items() if v[1]}},
             "fp64_roofline": {"legendre_synth": roof(st_syn["legendre_synth"][0]),
                               "legendre_anal": roof(st_ana["legendre_anal"][0]),
                               "work": "7 flops per (l, m, ring-pair) step, nominal full triangle S = %d" % S},
             "input": inp}
        if grid == sht.GRID_GAUSS_LEGENDRE:
            d = (back - alm).abs().max().item() / alm.abs().pow(2).mean().sqrt().item()
            r["round_trip_err"] = {"max_abs_over_rms": d, "bar": 1e-12,
                                   "input": "uniform a_lm in (-1, 1) (the paper's accuracy input)"}
        out[name] = r
        del alm, mp, back
        plan.close()
    del flush
    torch.cuda.empty_cache()
    out["form"] = "plain FP64, 1 map per call, lmax = mmax = 2048, median of %d repetitions after an L2 flush" % reps
    return out


def o1_leg(lmax=64, nside=32):
    """The oracle's exact pixel-by-pixel form (eqs. alm2mapDef / map2almDef with lambda recomputed
    per pixel), single-threaded, at HEALPix Nside 32, lmax 64, one map: seconds per transform."""
    import oracle
    from oracle import geometry
    from paper_1106_0159_gb300 import inputs

    oracle.build()
    geom = geometry.healpix(nside)
    a0 = inputs.gaussian_alm(lmax, lmax, seed=7)[0]
    old = oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        s0 = oracle.alm2map_exact(geom, a0, lmax, lmax)
        t1 = time.perf_counter()
        oracle.map2alm_exact(geom, s0, lmax, lmax)
        t2 = time.perf_counter()
    finally:
        oracle.set_threads(old)
    return {"alm2map_s": t1 - t0, "map2alm_s": t2 - t1, "round_trip_maps_per_s": 1.0 / (t2 - t0), "cores": 1,
            "cpu_model": cpu_model(), "form": "oracle O1 (pixel by pixel), one thread, HEALPix Nside %d, lmax %d, "
                                            "1 map" % (nside, lmax)}


def batch_leg(a, rep, local_rank):
    """The batched form: `--batch-maps` maps, each with lmax drawn from {512, 1024, 2048} (HEALPix
    nside = lmax/2) and alm2map or map2alm with probability 1/2.  Plain FP64: one persistent launch
    per stage and direction (tiles of all plans from one longest-first queue; the two directions on
    two streams of one CUDA graph), batch knobs autotuned first.  Beside it, and for the precision
    form, a CUDA graph of one library call per (lmax, direction) with the per-call knobs autotuned.
    Replays and eager calls are timed with CUDA events, `--steps` times each after one warm-up."""
    import functools

    import numpy as np
    import torch

    from paper_1106_0159_gb300 import autotune, batch, inputs, sht

    g = np.random.Generator(np.random.PCG64(rep.seed(5151)))
    lmaxes = [512, 1024, 2048]
    count = {}
    for _ in range(a.batch_maps):
        key = (lmaxes[int(g.integers(len(lmaxes)))], batch.ALM2MAP if g.random() < 0.5 else batch.MAP2ALM)
        count[key] = count.get(key, 0) + 1
    gen = torch.Generator(device="cuda")
    out = {"maps": a.batch_maps, "calls": {"%s lmax=%d" % (d, L): n for (L, d), n in sorted(count.items())}}
    for mode, name in ((sht.MODE_FP64, "fp64"), (sht.MODE_SPLIT_BF16, "precision")):
        gen.manual_seed(rep.seed(5152))
        plans = {}
        for L in lmaxes:
            plans[L] = sht.Plan(sht.healpix_geometry(L // 2), L, L, grid=sht.GRID_HEALPIX)
            plans[L].set_mode(mode)
        jobs = []
        for (L, d), n in sorted(count.items()):
            p = plans[L]
            if d == batch.ALM2MAP:
                lv, mv = inputs.lm_arrays(L, L)
                cl = 1.0 / (lv * (lv + 1.0) + 1.0)
                sd = torch.from_numpy(np.where(mv == 0, np.sqrt(cl), np.sqrt(cl / 2.0))).cuda()
                mnz = torch.from_numpy(mv != 0).cuda()
                x = torch.complex(torch.randn((n, p.nalm), dtype=torch.float64, device="cuda", generator=gen) * sd,
                                  torch.randn((n, p.nalm), dtype=torch.float64, device="cuda", generator=gen) * sd * mnz)
                y = torch.empty((n, p.npix), dtype=torch.float64, device="cuda")
            else:
                x = torch.randn((n, p.npix), dtype=torch.float64, device="cuda", generator=gen)
                y = torch.empty((n, p.nalm), dtype=torch.complex128, device="cuda")
            jobs.append(batch.Job(p, d, x, y))
        tuner = autotune.Autotuner(timer=functools.partial(autotune.cuda_timer, reps=1))
        t0 = time.perf_counter()
        recs = [tuner.tune(j.plan, j.direction, j.src, j.dst) for j in jobs]
        tune_s = time.perf_counter() - t0
        b = batch.GraphBatch(jobs, nstreams=2)
        t0 = time.perf_counter()
        b.capture()
        capture_s = time.perf_counter() - t0
        stream = torch.cuda.current_stream()

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            rep.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return rep.max_over_ranks(e0.elapsed_time(e1), device="cuda") / a.steps

        def eager():
            b.run_eager(b.streams)
            for st in b.streams:
                stream.wait_stream(st)

        g_ms = timed(b.replay)
        e_ms = timed(eager)
        res = {"graph_of_calls_ms": g_ms, "graph_of_calls_maps_per_s": a.batch_maps / (g_ms * 1e-3),
               "eager_ms": e_ms, "eager_maps_per_s": a.batch_maps / (e_ms * 1e-3),
               "tune_s": tune_s, "capture_s": capture_s,
               "tuned": {"%s lmax=%d" % (j.direction, j.plan.lmax): {"knobs": r["knobs"], "ms": r["ms"],
                                                                    "default_ms": r["default_ms"]}
                         for j, r in zip(jobs, recs)}}
        del b
        if mode == sht.MODE_FP64:
            # the persistent form: one launch per stage and direction, tiles of every plan from one
            # queue, longest first; the batch knobs (tile shapes, persistent grids) tuned first
            pb = batch.PersistentBatch(jobs)
            t0 = time.perf_counter()
            cache = {}
            ptuned = {d: autotune.tune_batch(bb, d, cache=cache, passes=1, timer=functools.partial(
                autotune.batch_timer, reps=1), key=autotune.batch_key([(j.plan, j.src) for j in jobs
                                                                       if j.direction == d], d))
                      for d, bb in pb.batches}
            ptune_s = time.perf_counter() - t0
            pb.capture()
            p_ms = timed(pb.replay)
            res.update({"persistent_ms": p_ms, "maps_per_s": a.batch_maps / (p_ms * 1e-3), "persistent_tune_s": ptune_s,
                        "persistent_tuned": {d: {"knobs": r["knobs"], "ms": r["ms"], "default_ms": r["default_ms"]}
                                             for d, r in ptuned.items()},
                        "tiles": {d: {"legendre": bb.tiles(0), "ring": bb.tiles(1)} for d, bb in pb.batches},
                        "form": "persistent: one launch per stage and direction, longest-first tile queue, both "
                                "directions on two streams of one CUDA graph"})
            pb.close()
        else:
            res.update({"maps_per_s": res["graph_of_calls_maps_per_s"],
                        "form": "graph of calls: one library call per (lmax, direction) on 2 streams of one CUDA "
                                "graph (the tensor-core kernels have no persistent multi-plan form)"})
        res["device_status"] = max(p.device_status() for p in plans.values())
        out[name] = res
        del jobs
        for p in plans.values():
            p.close()
        torch.cuda.empty_cache()
    out["precision_over_fp64"] = out["precision"]["maps_per_s"] / out["fp64"]["maps_per_s"]
    out["persistent_over_graph_of_calls_fp64"] = out["fp64"]["maps_per_s"] / out["fp64"]["graph_of_calls_maps_per_s"]
    return out


def serve_grid():
    """The serving trace's band limits: 16 values log-uniform between 256 and 4096, rounded to even
    (nside = lmax / 2), most of them not powers of two."""
    return [2 * int(round(128 * 16 ** (k / 15))) for k in range(16)]


def serve_leg(a, rep, local_rank):
    """The serving trace of the benchmark's configuration 5: `--serve-requests` requests, lmax drawn
    uniformly from serve_grid() (log-uniform over [256, 4096]) on HEALPix nside = lmax/2, 1-32 maps
    each, alm2map or map2alm with probability 1/2, inputs a C_l-shaped Gaussian a_lm or unit white
    noise, resident on the device before they arrive (one 32-map input per grid and direction,
    requests take its first maps).  Served twice: by the continuous-batching server in the precision
    form on two streams, and by the plain FP64 path one request per call in arrival order.  First
    both at saturation (every request at t = 0: capacity, maps/s), then both under Poisson arrivals
    at 80 % of the plain path's measured capacity (p50/p99 latency = completion - arrival)."""
    import numpy as np
    import torch

    from paper_1106_0159_gb300 import inputs, serve, sht

    g = np.random.Generator(np.random.PCG64(rep.seed(4242)))
    grid = serve_grid()
    spec = []
    for _ in range(a.serve_requests):
        L = grid[int(g.integers(len(grid)))]
        spec.append((serve.ALM2MAP if g.random() < 0.5 else serve.MAP2ALM, L, L // 2, int(g.integers(1, 33))))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(rep.seed(4243))
    pools = {}
    for d, L, ns, n in spec:
        if (d, L) in pools:
            continue
        if d == serve.ALM2MAP:
            l, m = inputs.lm_arrays(L, L)
            cl = 1.0 / (l * (l + 1.0) + 1.0)
            sd = torch.from_numpy(np.where(m == 0, np.sqrt(cl), np.sqrt(cl / 2.0))).cuda()
            mnz = torch.from_numpy(m != 0).cuda()
            re = torch.randn((32, sd.numel()), dtype=torch.float64, device="cuda", generator=gen) * sd
            im = torch.randn((32, sd.numel()), dtype=torch.float64, device="cuda", generator=gen) * sd * mnz
            pools[(d, L)] = torch.complex(re, im)
        else:
            pools[(d, L)] = torch.randn((32, 12 * (L // 2) ** 2), dtype=torch.float64, device="cuda", generator=gen)
    datas = [pools[(d, L)][:n] for d, L, ns, n in spec]
    torch.cuda.synchronize()
    keys = sorted(set((ns, L) for _, L, ns, _ in spec))
    nmaps = sum(n for *_, n in spec)
    mean_maps = nmaps / max(len(spec), 1)

    def run(mode, nstreams, batching, offsets, label):
        be = serve.TorchBackend(mode=mode, nstreams=nstreams, budget_fraction=0.8)
        warm_s = be.warm(keys, max_maps=32)
        srv = serve.Server(be, max_batch_maps=32, nstreams=nstreams, batching=batching, keep_results=False)
        trace = [(t, serve.Request(d, L, ns, x, n)) for t, (d, L, ns, n), x in zip(offsets, spec, datas)]
        rep.barrier()
        clocks = ClockSampler(local_rank)
        clocks.start()
        srv.run_trace(trace, timeout=1200)
        torch.cuda.synchronize()
        st = srv.stats()
        st["clocks"] = clocks.stop()
        st["plan_warm_s"] = warm_s
        st["device_status"] = max(be.plan(k).device_status() for k in keys)
        st["run"] = label
        be.close()
        return st

    zero = [0.0] * len(spec)
    plain_sat = run(sht.MODE_FP64, 1, False, zero, "plain, saturated")
    served_sat = run(sht.MODE_SPLIT_BF16, 2, True, zero, "served, saturated")
    rate = 0.8 * plain_sat["maps_per_s"] / mean_maps   # requests per second
    offsets = [t for t, _ in serve.poisson_trace(rate, len(spec), lambda i: i, seed=rep.seed(4244))]
    plain_ol = run(sht.MODE_FP64, 1, False, offsets, "plain, Poisson at 80 % of plain capacity")
    served_ol = run(sht.MODE_SPLIT_BF16, 2, True, offsets, "served, Poisson at 80 % of plain capacity")
    del datas, pools
    torch.cuda.empty_cache()
    return {"trace": "%d requests (%d maps), lmax uniform over %s (log-uniform in [256, 4096], even; HEALPix "
                     "nside = lmax/2), 1-32 maps each, alm2map or map2alm with probability 1/2; inputs resident "
                     "on the device" % (len(spec), nmaps, grid),
            "offered_rate_per_s": rate, "offered_load": "80 % of the plain path's saturated capacity",
            "served": {"saturated": served_sat, "open_loop": served_ol},
            "plain": {"saturated": plain_sat, "open_loop": plain_ol},
            "maps_per_s": {"served": served_sat["maps_per_s"], "plain": plain_sat["maps_per_s"]},
            "p50_ms": {"served": served_ol["p50_ms"], "plain": plain_ol["p50_ms"]},
            "p99_ms": {"served": served_ol["p99_ms"], "plain": plain_ol["p99_ms"]},
            "served_over_plain_maps_per_s": served_sat["maps_per_s"] / plain_sat["maps_per_s"],
            "served_form": "continuous batching, up to 32 maps of one plan and direction per call, 2 streams, "
                           "precision form",
            "plain_form": "one request per call in arrival order, 1 stream, plain FP64"}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    return ours_arm(a, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
