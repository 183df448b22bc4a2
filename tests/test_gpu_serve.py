"""The continuous-batching server on the GPU: every request's result is the same alone (one call
on its own plan) and when served in a mix of requests batched together and overlapping on two
streams.  Plain FP64 form: bitwise.  Precision form: within its bar (1e-9 of the RMS)."""
import numpy as np
import pytest

from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = [(64, 128), (128, 256)]   # (nside, lmax): both have non-polar ring blocks (tensor-core path)


def rel(x, ref):
    return float(torch.max(torch.abs(x - ref)) / torch.sqrt(torch.mean(torch.abs(ref) ** 2)))


def _requests(backend, seed):
    from paper_1106_0159_gb300.serve import ALM2MAP, MAP2ALM, Request
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(14):
        nside, lmax = KEYS[int(g.integers(len(KEYS)))] if i >= 3 else KEYS[0]
        direction = ALM2MAP if (i < 3 or g.random() < 0.5) else MAP2ALM   # the first three share a batch
        nmaps = int(g.integers(1, 5))
        p = backend.plan((nside, lmax), 0)
        if direction == ALM2MAP:
            x = inputs.gaussian_alm(lmax, lmax, seed=1000 + i, nmaps=nmaps)
        else:
            x = inputs.white_map(p.npix, seed=1000 + i, nmaps=nmaps)
        out.append(Request(direction, lmax, nside, torch.from_numpy(x).cuda(), nmaps))
    return out


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "split_bf16"])
def test_served_equals_alone(mode):
    from paper_1106_0159_gb300.serve import ALM2MAP, Server, TorchBackend
    be = TorchBackend(mode=mode, nstreams=2)
    be.warm(KEYS, max_maps=8)
    reqs = _requests(be, seed=7 + mode)

    alone = []
    for r in reqs:   # one call per request, on the slot-0 plan, default stream
        p = be.plan(r.key, 0)
        alone.append((p.alm2map(r.data) if r.direction == ALM2MAP else p.map2alm(r.data)).clone())
    torch.cuda.synchronize()

    srv = Server(be, max_batch_maps=8, nstreams=2)
    for r in reqs[:6]:
        srv.submit(r)
    srv.poll()                                  # two batches go out on the two streams
    assert len(srv.running) == 2
    for r in reqs[6:]:                          # the rest arrive while those run
        srv.submit(r)
        srv.poll()
    srv.drain(timeout=120)
    torch.cuda.synchronize()

    assert len(srv.completed) == len(reqs) and not srv.dropped
    assert srv.nbatches < len(reqs)            # some requests shared a batch
    for i in range(len(KEYS)):
        for slot in range(2):
            assert be.plan(KEYS[i], slot).device_status() == 0
    worst = 0.0
    for r, a in zip(reqs, alone):
        assert r.status == "done" and r.result.shape == a.shape
        if mode == 0:
            assert torch.equal(r.result, a), r.rid
        else:
            e = rel(r.result, a)
            worst = max(worst, e)
            assert e <= 1e-9, (r.rid, e)
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    print("mode", mode, "worst served-vs-alone", worst, st)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "split_bf16"])
def test_caller_scratch_calls_match_and_check_their_scratch(mode):
    from paper_1106_0159_gb300 import sht
    p = sht.Plan(sht.healpix_geometry(64), 128, 128, grid=sht.GRID_HEALPIX)
    p.set_mode(mode)
    a = torch.from_numpy(inputs.gaussian_alm(128, 128, seed=93, nmaps=5)).cuda()
    m = p.alm2map(a)
    b = p.map2alm(m)
    scr = p.scratch(5)
    assert torch.equal(p.alm2map_ws(a, scr), m)
    assert torch.equal(p.map2alm_ws(m, scr), b)
    with pytest.raises(ValueError):                 # SHT_EINVAL
        p.alm2map_ws(a, p.scratch(1)[:16])          # too small
    with pytest.raises(ValueError):
        p.map2alm_ws(m, scr[8:])                    # not 256-byte aligned
    assert p.device_status() == 0
