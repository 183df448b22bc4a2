"""Autotuner for a plan's launch-tuning knobs (sht_plan_set_tuning).

For a key (grid, band limits, maps per call, mode, direction) it times every combination of the
knobs that the direction and mode use, one transform each (after a warm-up), with CUDA events on
the call's stream, keeps the fastest and caches it (in memory, and in a JSON file when a path is
given).  Every combination gives the same synthesis results and analysis results within rounding
(the FP64 ring sums change order with the slots per thread), so tuning only moves time.

The timer is injectable so that the search and the cache can be tested without a GPU.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Callable, Dict, List, Optional, Tuple

from . import sht

ALM2MAP, MAP2ALM = "alm2map", "map2alm"


def knobs_for(direction: str, mode: int) -> List[int]:
    """The knobs a transform of this direction and mode reads."""
    if direction == ALM2MAP:
        # precision form: tensor-core groups, and the FP64 kernel on polar slot blocks
        return [sht.TUNE_TC_MAPS, sht.TUNE_SYNTH_MAPS] if mode == sht.MODE_SPLIT_BF16 else [sht.TUNE_SYNTH_MAPS]
    if direction == MAP2ALM:
        # precision form: tensor-core or double-float kernel (the latter's maps per launch)
        return [sht.TUNE_PREC_ANAL, sht.TUNE_DF_MAPS] if mode == sht.MODE_SPLIT_BF16 else [sht.TUNE_ANAL_MAPS, sht.TUNE_ANAL_SLOTS]
    raise ValueError("unknown direction %r" % (direction,))


def candidates(direction: str, mode: int, nmaps: int) -> List[Dict[int, int]]:
    """Knob settings worth timing: values above the call's map count act like the map count, so
    only the smallest of those is kept; the double-float maps per launch matter only when the
    double-float analysis kernel is chosen."""
    ks = knobs_for(direction, mode)
    per_knob = []
    for k in ks:
        vals = sorted(sht.TUNE_VALUES[k])
        if k in (sht.TUNE_SYNTH_MAPS, sht.TUNE_ANAL_MAPS, sht.TUNE_DF_MAPS, sht.TUNE_TC_MAPS):
            keep = [v for v in vals if v < nmaps] + [min([v for v in vals if v >= nmaps] or [vals[-1]])]
            vals = sorted(set(keep))
        per_knob.append(vals)
    out = []
    for combo in itertools.product(*per_knob):
        c = dict(zip(ks, combo))
        if c.get(sht.TUNE_PREC_ANAL) == 1 and c[sht.TUNE_DF_MAPS] != per_knob[ks.index(sht.TUNE_DF_MAPS)][-1]:
            continue  # tensor-core analysis: the double-float grouping is unused, keep one setting
        out.append(c)
    return out


def plan_key(plan, nmaps: int, direction: str) -> str:
    return "nrings=%d npix=%d lmax=%d mmax=%d mode=%d nmaps=%d %s" % (
        plan.nrings, plan.npix, plan.lmax, plan.mmax, plan.mode, nmaps, direction)


def cuda_timer(plan, direction: str, src, dst, reps: int = 2) -> float:
    """Milliseconds of one transform (median of `reps` after one warm-up), CUDA events on the
    current stream."""
    import torch
    fn = plan.alm2map if direction == ALM2MAP else plan.map2alm
    fn(src, out=dst)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(src, out=dst)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


class Autotuner:
    def __init__(self, path: Optional[str] = None, timer: Callable = cuda_timer):
        self.path = path
        self.timer = timer
        self.cache: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def _save(self):
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    @staticmethod
    def _apply(plan, knobs: Dict[int, int]):
        for k, v in knobs.items():
            plan.set_tuning(int(k), int(v))

    def apply(self, plan, nmaps: int, direction: str) -> bool:
        """Set the cached best knobs for this key; False if the key was never tuned."""
        rec = self.cache.get(plan_key(plan, nmaps, direction))
        if rec is None:
            return False
        self._apply(plan, {int(k): v for k, v in rec["knobs"].items()})
        return True

    def tune(self, plan, direction: str, src, dst, force: bool = False) -> dict:
        """Time every candidate on (src -> dst), keep the fastest on the plan; returns the record
        {"knobs", "ms", "default_ms", "tried"}.  A cached key is applied without timing."""
        nmaps = int(src.shape[0]) if hasattr(src, "shape") and len(src.shape) > 1 else 1
        key = plan_key(plan, nmaps, direction)
        if not force and key in self.cache:
            self.apply(plan, nmaps, direction)
            return self.cache[key]
        ks = knobs_for(direction, plan.mode)
        default = {k: plan.tuning(k) for k in ks}
        tried: List[Tuple[Dict[int, int], float]] = []
        for cand in candidates(direction, plan.mode, nmaps):
            self._apply(plan, cand)
            tried.append((cand, float(self.timer(plan, direction, src, dst))))
        self._apply(plan, default)
        default_ms = float(self.timer(plan, direction, src, dst))
        best, best_ms = min(tried, key=lambda t: t[1])
        if default_ms <= best_ms:
            best, best_ms = default, default_ms
        self._apply(plan, best)
        rec = {"knobs": {str(k): v for k, v in best.items()}, "ms": best_ms, "default_ms": default_ms,
               "tried": [[{str(k): v for k, v in c.items()}, t] for c, t in tried]}
        self.cache[key] = rec
        self._save()
        return rec


# ---------------------------------------------------------------- the persistent batched form

def batch_knobs(direction: str) -> List[int]:
    """The batch knobs a direction reads: tile shapes (maps per tile, slots per thread) and the
    persistent grids (CTAs per SM of the Legendre and ring launches)."""
    if direction == ALM2MAP:
        return [sht.BATCH_SYNTH_MAPS, sht.BATCH_LEG_CTAS, sht.BATCH_RING_CTAS]
    if direction == MAP2ALM:
        return [sht.BATCH_ANAL_MAPS, sht.BATCH_ANAL_SLOTS, sht.BATCH_LEG_CTAS, sht.BATCH_RING_CTAS]
    raise ValueError("unknown direction %r" % (direction,))


def batch_key(jobs, direction: str) -> str:
    """Cache key of a batch: its (grid size, lmax, maps) jobs, the mode and the direction."""
    parts = sorted("%d:%d:%d:%d" % (j[0].npix, j[0].lmax, j[0].mode, int(j[1].shape[0])) for j in jobs)
    return "batch %s %s" % (direction, ",".join(parts))


def batch_timer(batch, reps: int = 2) -> float:
    """Milliseconds of one batch run (median of `reps` after one warm-up), CUDA events."""
    import torch
    batch.run()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune_batch(batch, direction: str, timer: Callable = batch_timer, cache: Optional[Dict[str, dict]] = None,
               key: Optional[str] = None, passes: int = 2) -> dict:
    """Coordinate search over the batch knobs: from the defaults, each knob in turn takes the
    fastest of its values with the others fixed, `passes` times over.  Returns {"knobs", "ms",
    "default_ms", "tried"}; with a cache and a key, a cached record is applied without timing."""
    if cache is not None and key is not None and key in cache:
        for k, v in cache[key]["knobs"].items():
            batch.set_tuning(int(k), int(v))
        return cache[key]
    ks = batch_knobs(direction)
    cur = {k: batch.tuning(k) for k in ks}
    default_ms = float(timer(batch))
    best_ms = default_ms
    tried = []
    for _ in range(max(1, passes)):
        for k in ks:
            for v in sht.BATCH_TUNE_VALUES[k]:
                if v == cur[k]:
                    continue
                batch.set_tuning(k, v)
                t = float(timer(batch))
                tried.append([{str(kk): (v if kk == k else cur[kk]) for kk in ks}, t])
                if t < best_ms:
                    best_ms, cur[k] = t, v
                batch.set_tuning(k, cur[k])
    rec = {"knobs": {str(k): v for k, v in cur.items()}, "ms": best_ms, "default_ms": default_ms, "tried": tried}
    if cache is not None and key is not None:
        cache[key] = rec
    return rec
