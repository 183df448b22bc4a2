"""The persistent batched form (sht_batch_*): transforms of uneven lmax and map counts, one
persistent launch per stage and direction with a longest-first tile queue.  Its results are the
one-plan calls' bit for bit (same kernels, same summation order), whatever the knobs, they match
the oracle on sampled rings and m of every lmax, and a CUDA-graph replay equals the eager run."""
import numpy as np
import pytest

import oracle
from oracle import geometry
from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LMAXES = (64, 96, 128)
SYN_MAPS = {64: 3, 96: 1, 128: 5}
ANA_MAPS = {64: 2, 96: 4, 128: 1}


def rel(x, ref):
    x, ref = np.asarray(x), np.asarray(ref)
    return float(np.max(np.abs(x - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


@pytest.fixture(scope="module")
def setup():
    from paper_1106_0159_gb300 import sht
    plans = {L: sht.Plan(sht.healpix_geometry(L // 2), L, L, grid=sht.GRID_HEALPIX) for L in LMAXES}
    for p in plans.values():
        p.set_tuning(sht.TUNE_ANAL_SLOTS, 4)   # the batch's default slots per thread
    syn, ana = [], []
    for L in LMAXES:
        p = plans[L]
        a = torch.from_numpy(inputs.gaussian_alm(L, L, seed=300 + L, nmaps=SYN_MAPS[L])).cuda()
        syn.append((p, a, torch.empty((SYN_MAPS[L], p.npix), dtype=torch.float64, device="cuda")))
        s = torch.from_numpy(inputs.white_map(p.npix, seed=400 + L, nmaps=ANA_MAPS[L])).cuda()
        ana.append((p, s, torch.empty((ANA_MAPS[L], p.nalm), dtype=torch.complex128, device="cuda")))
    yield sht, plans, syn, ana
    for p in plans.values():
        p.close()


def test_batch_equals_single_plan_calls_and_oracle(setup):
    sht, plans, syn, ana = setup
    bs = sht.Batch(sht.BATCH_ALM2MAP, syn)
    ba = sht.Batch(sht.BATCH_MAP2ALM, ana)
    bs.run()
    ba.run()
    torch.cuda.synchronize()
    for p, a, out in syn:
        assert torch.equal(out, p.alm2map(a))
    for p, s, out in ana:
        assert torch.equal(out, p.map2alm(s))
    # every (map group of 4, 2 or 1 maps, m, 128-slot block) of every plan is one tile
    def groups(n):
        return n // 4 + (n % 4) // 2 + (n % 2)
    want = sum(groups(SYN_MAPS[L]) * (L + 1) * ((plans[L].npairs + 127) // 128) for L in LMAXES)
    assert bs.tiles(0) == want
    # against the oracle on sampled rings and m of every lmax
    for p, a, out in syn:
        L = p.lmax
        geom = geometry.healpix(L // 2)
        rings = [0, 1, L // 4, p.nrings // 2, p.nrings - 1]
        off = geometry.ring_offsets(geom)
        for g in (0, SYN_MAPS[L] - 1):
            ref = oracle.alm2map_rings(geom, a[g].cpu().numpy(), L, L, rings)
            got = np.concatenate([out[g].cpu().numpy()[off[r]:off[r + 1]] for r in rings])
            assert rel(got, ref) < 1e-11
    for p, s, out in ana:
        L = p.lmax
        geom = geometry.healpix(L // 2)
        ms = [0, 1, L // 2, L]
        for g in (0, ANA_MAPS[L] - 1):
            refs = oracle.map2alm_ms(geom, s[g].cpu().numpy(), L, ms)
            b = out[g].cpu().numpy()
            got = np.concatenate([b[oracle.alm_index(L, m, m):oracle.alm_index(L, m, m) + L - m + 1] for m in ms])
            assert rel(got, np.concatenate(refs)) < 1e-11
    bs.close()
    ba.close()


def test_knobs_change_nothing(setup):
    sht, plans, syn, ana = setup
    bs = sht.Batch(sht.BATCH_ALM2MAP, syn)
    bs.run()
    torch.cuda.synchronize()
    want = [o.clone() for _, _, o in syn]
    for knob, vals in ((sht.BATCH_SYNTH_MAPS, (1, 2, 4)), (sht.BATCH_LEG_CTAS, (2, 16)),
                       (sht.BATCH_RING_CTAS, (1, 3))):
        for v in vals:
            bs.set_tuning(knob, v)
            for _, _, o in syn:
                o.zero_()
            bs.run()
            torch.cuda.synchronize()
            assert all(torch.equal(o, w) for (_, _, o), w in zip(syn, want)), (knob, v)
    with pytest.raises(ValueError):
        bs.set_tuning(sht.BATCH_SYNTH_MAPS, 3)
    bs.close()
    ba = sht.Batch(sht.BATCH_MAP2ALM, ana)
    ba.run()
    torch.cuda.synchronize()
    want = [o.clone() for _, _, o in ana]
    for knob, vals in ((sht.BATCH_ANAL_MAPS, (1, 2)), (sht.BATCH_LEG_CTAS, (4, 8)), (sht.BATCH_RING_CTAS, (2,))):
        for v in vals:
            ba.set_tuning(knob, v)
            ba.run()
            torch.cuda.synchronize()
            assert all(torch.equal(o, w) for (_, _, o), w in zip(ana, want)), (knob, v)
    ba.close()


def test_graph_replay_equals_eager_and_follows_new_inputs(setup):
    from paper_1106_0159_gb300 import batch
    sht, plans, syn, ana = setup
    jobs = [batch.Job(p, batch.ALM2MAP, a, o) for p, a, o in syn] + [batch.Job(p, batch.MAP2ALM, s, o)
                                                                      for p, s, o in ana]
    b = batch.PersistentBatch(jobs).capture()
    for j in jobs:
        j.dst.zero_()
    b.replay()
    torch.cuda.synchronize()
    for j in jobs:
        ref = j.plan.alm2map(j.src) if j.direction == batch.ALM2MAP else j.plan.map2alm(j.src)
        assert torch.equal(j.dst, ref)
    syn[0][1].mul_(-2.0)  # new inputs, written in place
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(syn[0][2], syn[0][0].alm2map(syn[0][1]))
    b.close()


def test_precision_form_plans_are_refused(setup):
    sht, plans, syn, ana = setup
    q = sht.Plan(sht.healpix_geometry(16), 32, 32)
    q.set_mode(sht.MODE_SPLIT_BF16)
    a = torch.zeros((1, q.nalm), dtype=torch.complex128, device="cuda")
    m = torch.zeros((1, q.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(sht.ShtError) as e:
        sht.Batch(sht.BATCH_ALM2MAP, [(q, a, m)])
    assert e.value.status == sht.SHT_EUNSUPPORTED
    q.close()
