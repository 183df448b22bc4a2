"""Host logic of the autotuner and of the CUDA-graph batch: candidate sets, the search with a fake
timer, the cache, and how jobs are dealt over streams (no GPU)."""
import json

import numpy as np
import pytest

from paper_1106_0159_gb300 import autotune, sht
from paper_1106_0159_gb300.batch import ALM2MAP, MAP2ALM, GraphBatch, Job, assign_streams


class FakePlan:
    def __init__(self, lmax=64, mode=sht.MODE_FP64, nrings=127, npix=12288):
        self.lmax = self.mmax = lmax
        self.mode = mode
        self.nrings, self.npix = nrings, npix
        self.knobs = {sht.TUNE_SYNTH_MAPS: 4, sht.TUNE_ANAL_MAPS: 2, sht.TUNE_ANAL_SLOTS: 4,
                      sht.TUNE_DF_MAPS: 8, sht.TUNE_TC_MAPS: 16, sht.TUNE_PREC_ANAL: 1}

    def set_tuning(self, k, v):
        assert v in sht.TUNE_VALUES[k]
        self.knobs[k] = v

    def tuning(self, k):
        return self.knobs[k]


def test_candidates_cover_the_knobs_of_each_form():
    assert autotune.knobs_for(ALM2MAP, sht.MODE_FP64) == [sht.TUNE_SYNTH_MAPS]
    assert autotune.knobs_for(MAP2ALM, sht.MODE_FP64) == [sht.TUNE_ANAL_MAPS, sht.TUNE_ANAL_SLOTS]
    assert autotune.knobs_for(MAP2ALM, sht.MODE_SPLIT_BF16) == [sht.TUNE_PREC_ANAL, sht.TUNE_DF_MAPS]
    c = autotune.candidates(ALM2MAP, sht.MODE_FP64, 16)
    assert [x[sht.TUNE_SYNTH_MAPS] for x in c] == [1, 2, 4]
    # values above the map count collapse to the smallest of them
    c = autotune.candidates(ALM2MAP, sht.MODE_FP64, 1)
    assert [x[sht.TUNE_SYNTH_MAPS] for x in c] == [1]
    c = autotune.candidates(MAP2ALM, sht.MODE_SPLIT_BF16, 6)
    assert [(x[sht.TUNE_PREC_ANAL], x[sht.TUNE_DF_MAPS]) for x in c] == [(0, 4), (0, 8), (1, 8)]
    c = autotune.candidates(MAP2ALM, sht.MODE_FP64, 16)
    assert len(c) == 4 and {(x[sht.TUNE_ANAL_MAPS], x[sht.TUNE_ANAL_SLOTS]) for x in c} == {(1, 1), (1, 4), (2, 1), (2, 4)}
    assert len(autotune.candidates(ALM2MAP, sht.MODE_SPLIT_BF16, 16)) == 2 * 3
    with pytest.raises(ValueError):
        autotune.knobs_for("sideways", 0)


def test_tune_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(plan, direction, src, dst):
        calls.append(dict(plan.knobs))
        # fastest: 1 map per launch, 4 slots per thread
        return 10.0 - (plan.knobs[sht.TUNE_ANAL_SLOTS] == 4) * 3 - (plan.knobs[sht.TUNE_ANAL_MAPS] == 1) * 2

    path = str(tmp_path / "tune.json")
    t = autotune.Autotuner(path=path, timer=timer)
    p = FakePlan()
    src = np.zeros((16, 10))
    rec = t.tune(p, MAP2ALM, src, None)
    assert rec["knobs"] == {str(sht.TUNE_ANAL_MAPS): 1, str(sht.TUNE_ANAL_SLOTS): 4}
    assert p.knobs[sht.TUNE_ANAL_MAPS] == 1 and p.knobs[sht.TUNE_ANAL_SLOTS] == 4
    assert rec["ms"] == 5.0 and rec["default_ms"] == 7.0 and len(rec["tried"]) == 4
    n = len(calls)
    # cached: applied without timing, also from a new tuner reading the file
    p2 = FakePlan()
    t2 = autotune.Autotuner(path=path, timer=timer)
    assert t2.tune(p2, MAP2ALM, src, None)["ms"] == 5.0 and len(calls) == n
    assert p2.knobs[sht.TUNE_ANAL_MAPS] == 1
    assert json.load(open(path))
    # another key (map count) is tuned anew
    t2.tune(FakePlan(), MAP2ALM, np.zeros((3, 10)), None)
    assert len(calls) > n
    assert not t2.apply(FakePlan(lmax=128), 16, MAP2ALM)


def test_tune_keeps_default_when_nothing_is_faster():
    t = autotune.Autotuner(timer=lambda plan, d, s, o: 1.0)
    p = FakePlan()
    rec = t.tune(p, ALM2MAP, np.zeros((16, 4)), None)
    assert rec["knobs"] == {str(sht.TUNE_SYNTH_MAPS): 4} and p.knobs[sht.TUNE_SYNTH_MAPS] == 4


class Arr:
    def __init__(self, n):
        self.shape = (n, 8)


def test_streams_keep_a_plans_jobs_together_and_balance_work():
    a, b, c = FakePlan(lmax=2048), FakePlan(lmax=1024), FakePlan(lmax=512)
    jobs = [Job(a, ALM2MAP, Arr(40), None), Job(b, MAP2ALM, Arr(40), None), Job(a, MAP2ALM, Arr(40), None),
            Job(c, ALM2MAP, Arr(40), None), Job(b, ALM2MAP, Arr(40), None)]
    lanes = assign_streams(jobs, 2)
    assert len(lanes) == 2
    where = {}
    for i, ln in enumerate(lanes):
        for j in ln:
            where.setdefault(id(j.plan), set()).add(i)
    assert all(len(v) == 1 for v in where.values())     # one stream per plan
    assert [j.direction for j in lanes[0]] == [ALM2MAP, MAP2ALM]   # plan a alone (most work), in order
    assert {id(j.plan) for j in lanes[1]} == {id(b), id(c)}
    assert len(assign_streams(jobs, 8)) == 3               # no empty streams
    with pytest.raises(ValueError):
        GraphBatch([Job(a, "sideways", Arr(1), None)])
    with pytest.raises(RuntimeError):
        GraphBatch(jobs).replay()


class _FakeBatch:
    """Stands in for sht.Batch: knob values and a cost surface with one best point."""

    def __init__(self, best):
        from paper_1106_0159_gb300 import sht
        self.k = {sht.BATCH_SYNTH_MAPS: 4, sht.BATCH_LEG_CTAS: 8, sht.BATCH_RING_CTAS: 4, sht.BATCH_ANAL_MAPS: 2,
                  sht.BATCH_ANAL_SLOTS: 4}
        self.best = best
        self.sets = 0

    def tuning(self, knob):
        return self.k[knob]

    def set_tuning(self, knob, value):
        from paper_1106_0159_gb300 import sht
        assert value in sht.BATCH_TUNE_VALUES[knob]
        self.k[knob] = value
        self.sets += 1

    def cost(self):
        return 10.0 + sum(abs(self.k[k] - v) for k, v in self.best.items())


def test_tune_batch_finds_the_best_tile_shapes_and_grids():
    from paper_1106_0159_gb300 import sht
    best = {sht.BATCH_SYNTH_MAPS: 2, sht.BATCH_LEG_CTAS: 16, sht.BATCH_RING_CTAS: 2}
    b = _FakeBatch(best)
    rec = autotune.tune_batch(b, autotune.ALM2MAP, timer=lambda bb: bb.cost())
    assert rec["ms"] == 10.0 and rec["default_ms"] > 10.0
    assert {int(k): v for k, v in rec["knobs"].items()} == best
    assert all(b.k[k] == v for k, v in best.items())          # left at the best setting
    cache = {}
    b2 = _FakeBatch(best)
    autotune.tune_batch(b2, autotune.ALM2MAP, timer=lambda bb: bb.cost(), cache=cache, key="k")
    b3 = _FakeBatch(best)
    again = autotune.tune_batch(b3, autotune.ALM2MAP, timer=lambda bb: 1e9, cache=cache, key="k")
    assert again is cache["k"] and all(b3.k[k] == v for k, v in best.items())   # cached: applied, not timed
    assert autotune.batch_knobs(autotune.MAP2ALM) == [sht.BATCH_ANAL_MAPS, sht.BATCH_ANAL_SLOTS, sht.BATCH_LEG_CTAS,
                                                      sht.BATCH_RING_CTAS]
