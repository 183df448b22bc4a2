"""Batched form on the GPU: a mixed batch (three band limits, both directions, several map counts)
replayed as one CUDA graph gives the eager results bit for bit, also after its inputs are
rewritten in place; every launch-tuning setting gives the same synthesis bit for bit and the same
analysis within rounding; the autotuner leaves a plan that still matches."""
import numpy as np
import pytest

from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = [(32, 64), (64, 128), (128, 256)]  # (nside, lmax)


def rel(x, ref):
    return float(torch.max(torch.abs(x - ref)) / torch.sqrt(torch.mean(torch.abs(ref) ** 2)))


def _plans(mode):
    from paper_1106_0159_gb300 import sht
    out = {}
    for nside, L in KEYS:
        p = sht.Plan(sht.healpix_geometry(nside), L, L, grid=sht.GRID_HEALPIX)
        p.set_mode(mode)
        out[(nside, L)] = p
    return out


def _jobs(plans, seed):
    from paper_1106_0159_gb300.batch import ALM2MAP, MAP2ALM, Job
    g = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for i, (key, p) in enumerate(sorted(plans.items())):
        for direction in (ALM2MAP, MAP2ALM):
            n = int(g.integers(1, 6))
            if direction == ALM2MAP:
                x = torch.from_numpy(inputs.gaussian_alm(p.lmax, p.mmax, seed=seed + 10 * i, nmaps=n)).cuda()
                y = torch.empty((n, p.npix), dtype=torch.float64, device="cuda")
            else:
                x = torch.from_numpy(inputs.white_map(p.npix, seed=seed + 10 * i + 1, nmaps=n)).cuda()
                y = torch.empty((n, p.nalm), dtype=torch.complex128, device="cuda")
            jobs.append(Job(p, direction, x, y))
    return jobs


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "split_bf16"])
def test_graph_replay_equals_eager(mode):
    from paper_1106_0159_gb300.batch import GraphBatch
    plans = _plans(mode)
    jobs = _jobs(plans, seed=300 + mode)
    b = GraphBatch(jobs, nstreams=2)
    b.run_eager()
    torch.cuda.synchronize()
    eager = [j.dst.clone() for j in jobs]
    b.capture()
    for j in jobs:
        j.dst.zero_()
    b.replay()
    torch.cuda.synchronize()
    for j, e in zip(jobs, eager):
        assert torch.equal(j.dst, e)
    # new inputs written in place: the replay gives what eager calls on them give
    for j in jobs:
        j.src.mul_(-0.5)
    b.replay()
    torch.cuda.synchronize()
    replayed = [j.dst.clone() for j in jobs]
    b.run_eager()
    torch.cuda.synchronize()
    for j, r in zip(jobs, replayed):
        assert torch.equal(j.dst, r)
    for p in plans.values():
        assert p.device_status() == 0


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "split_bf16"])
def test_every_tuning_gives_the_same_result(mode):
    from paper_1106_0159_gb300 import autotune, sht
    from paper_1106_0159_gb300.batch import ALM2MAP, MAP2ALM
    p = sht.Plan(sht.healpix_geometry(128), 256, 256, grid=sht.GRID_HEALPIX)
    p.set_mode(mode)
    a = torch.from_numpy(inputs.gaussian_alm(256, 256, seed=71, nmaps=11)).cuda()
    s = torch.from_numpy(inputs.white_map(p.npix, seed=72, nmaps=11)).cuda()
    ref_map = p.alm2map(a)
    ref_alm = p.map2alm(s)
    for cand in autotune.candidates(ALM2MAP, mode, 11):
        for k, v in cand.items():
            p.set_tuning(k, v)
        got = p.alm2map(a)
        # FP64: the same arithmetic per map; precision form: the MMA width (16 or 32 columns)
        # changes with the maps per launch, the per-column sums should not
        assert torch.equal(got, ref_map) or (mode == sht.MODE_SPLIT_BF16 and rel(got, ref_map) < 1e-14), cand
    for cand in autotune.candidates(MAP2ALM, mode, 11):
        for k, v in cand.items():
            p.set_tuning(k, v)
        got = p.map2alm(s)
        if mode == sht.MODE_SPLIT_BF16:
            if cand[sht.TUNE_PREC_ANAL] == 1:      # tensor cores (the default): one launch of 11 maps
                assert torch.equal(got, ref_alm), cand
            else:                                   # double-float: within the precision bar of it
                assert rel(got, ref_alm) < 1e-9, cand
        else:
            assert rel(got, ref_alm) < 1e-13, cand
    assert p.device_status() == 0


def test_autotuner_on_the_gpu(tmp_path):
    from paper_1106_0159_gb300 import autotune, sht
    from paper_1106_0159_gb300.batch import ALM2MAP, MAP2ALM
    p = sht.Plan(sht.healpix_geometry(64), 128, 128, grid=sht.GRID_HEALPIX)
    a = torch.from_numpy(inputs.gaussian_alm(128, 128, seed=81, nmaps=6)).cuda()
    m = torch.empty((6, p.npix), dtype=torch.float64, device="cuda")
    back = torch.empty((6, p.nalm), dtype=torch.complex128, device="cuda")
    ref_map = p.alm2map(a).clone()
    ref_back = p.map2alm(ref_map).clone()
    t = autotune.Autotuner(path=str(tmp_path / "t.json"))
    r1 = t.tune(p, ALM2MAP, a, m)
    r2 = t.tune(p, MAP2ALM, ref_map, back)
    assert r1["ms"] > 0 and r2["ms"] > 0 and len(r1["tried"]) == 3 and len(r2["tried"]) == 4
    assert torch.equal(p.alm2map(a), ref_map)
    assert rel(p.map2alm(ref_map), ref_back) < 1e-13
