"""The m/ring-sharded transform on one GPU: every rank's stages are the library's (an m-list plan
over every ring for the Legendre step, a plan over the rank's rings for the ring step), the ranks
run in one process and the Delta transpose is a set of copies.  Together they must give what the
plain FP64 transforms give, and the m-list plan alone must compute only its m."""
import numpy as np
import pytest

from oracle import geometry
from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(x, ref):
    return float(np.max(np.abs(x - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


def test_mlist_plan_computes_only_its_m():
    from paper_1106_0159_gb300 import sht
    geom = geometry.healpix(16)
    L = 32
    p = sht.Plan(geom, L, L)
    a = torch.from_numpy(inputs.gaussian_alm(L, L, seed=91)).cuda()
    full = p.legendre_synth(a).cpu().numpy()
    ms = [0, 5, 31, 32]
    p.set_mlist(ms)
    part = p.legendre_synth(a).cpu().numpy()
    assert np.array_equal(part[:, :, ms], full[:, :, ms])
    others = [m for m in range(L + 1) if m not in ms]
    assert np.all(part[:, :, others] == 0.0)
    s = p.alm2map(a)  # the m-list synthesis reads a_lm of the listed m only
    b = p.map2alm(s).cpu().numpy()[0]
    lv, mv = inputs.lm_arrays(L, L)
    assert np.all(b[~np.isin(mv, ms)] == 0.0)
    with pytest.raises(ValueError):
        p.set_mlist([3, 3])
    with pytest.raises(ValueError):
        p.set_mlist([L + 1])
    p.set_mode(sht.MODE_SPLIT_BF16)
    with pytest.raises(sht.ShtError) as e:
        p.alm2map(a)
    assert e.value.status == sht.SHT_EUNSUPPORTED
    p.set_mode(sht.MODE_FP64)
    p.set_mlist(None)
    assert np.array_equal(p.legendre_synth(a).cpu().numpy(), full)
    p.close()


@pytest.mark.parametrize("nranks", [2, 3])
def test_sharded_loopback_equals_plain(nranks):
    from paper_1106_0159_gb300 import sharded, sht
    nside, L = 64, 128
    geom = sht.healpix_geometry(nside)
    part = sharded.Partition(geom[0], geom[1], L, nranks)
    stages = [sharded.LibraryStages(part, r, geom, L, grid=sht.GRID_HEALPIX) for r in range(nranks)]
    plain = sht.Plan(geom, L, L, grid=sht.GRID_HEALPIX)
    a = torch.from_numpy(inputs.gaussian_alm(L, L, seed=92, nmaps=2)).cuda()
    want = plain.alm2map(a).cpu().numpy()
    pix = sharded.alm2map_loopback(part, stages, a)
    off = np.concatenate([[0], np.cumsum(geom[0])])
    got = np.zeros_like(want)
    for r in range(nranks):
        o = 0
        px = pix[r].cpu().numpy()
        for ring in part.rings[r]:
            n = int(off[ring + 1] - off[ring])
            got[:, off[ring]:off[ring + 1]] = px[:, o:o + n]
            o += n
    assert rel(got, want) < 1e-14
    # analysis of the plain map, sharded by rings on the way in and by m on the way out
    s = torch.from_numpy(want).cuda()
    per = []
    for r in range(nranks):
        idx = np.concatenate([np.arange(off[ring], off[ring + 1]) for ring in part.rings[r]])
        per.append(s[:, torch.as_tensor(idx, device="cuda")].contiguous())
    alms = sharded.map2alm_loopback(part, stages, per)
    got = sum(x.cpu().numpy() for x in alms)
    assert rel(got, plain.map2alm(s).cpu().numpy()) < 1e-14
    for st in stages:
        st.close()
    plain.close()
