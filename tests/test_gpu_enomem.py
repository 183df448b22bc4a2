"""Allocation failures, injected on the host (sht_debug_fail_allocations_after: the library's
next device allocation fails as if the device were full, without a real out-of-memory condition):
every failure point of plan creation, of the precision-form and spin tables and of the workspace
returns SHT_ENOMEM, leaves no device memory behind, and leaves the plan usable."""
import pytest

from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _inject(n):
    from paper_1106_0159_gb300 import sht
    return sht.load().sht_debug_fail_allocations_after(n)


def test_every_allocation_failure_is_enomem_without_leak():
    from paper_1106_0159_gb300 import sht
    geom = sht.healpix_geometry(16)
    L = 32
    # every kernel used below runs once first: loading a kernel's module on its first launch
    # reserves device memory of its own, which is not the library's
    w = sht.Plan(geom, L, L)
    a0 = torch.from_numpy(inputs.gaussian_alm(L, L, seed=4)).cuda()
    w.map2alm(w.alm2map(a0))
    w.set_mode(sht.MODE_SPLIT_BF16)
    w.map2alm(w.alm2map(a0))
    w.set_mode(sht.MODE_FP64)
    w.alm2map_spin(torch.zeros((1, 2, w.nalm), dtype=torch.complex128, device="cuda"))
    w.close()
    del a0
    torch.cuda.synchronize()
    base = _free()
    k = 0
    while True:
        _inject(k)
        try:
            p = sht.Plan(geom, L, L)
        except sht.ShtError as e:
            _inject(-1)
            assert e.status == sht.SHT_ENOMEM, (k, e)
            assert _free() == base, k
            k += 1
            assert k < 100
            continue
        finally:
            _inject(-1)
        break
    assert k >= 10  # plan creation makes that many allocations
    a = torch.from_numpy(inputs.gaussian_alm(L, L, seed=5)).cuda()
    want = p.alm2map(a).clone()
    out = torch.empty_like(want)   # preallocated, so that the checks below allocate nothing
    with_ws = _free()
    # precision-form tables: every failure point, then the plan still runs in FP64 and switches later
    k = 0
    while True:
        _inject(k)
        try:
            p.set_mode(sht.MODE_SPLIT_BF16)
        except sht.ShtError as e:
            _inject(-1)
            assert e.status == sht.SHT_ENOMEM
            assert p.mode == sht.MODE_FP64 and _free() == with_ws
            p.alm2map(a, out=out)
            assert torch.equal(out, want)
            k += 1
            assert k < 20
            continue
        finally:
            _inject(-1)
        break
    assert k >= 2
    p.set_mode(sht.MODE_FP64)
    # a transform whose workspace must grow: ENOMEM, nothing enqueued, then it works
    a8 = torch.from_numpy(inputs.gaussian_alm(L, L, seed=6, nmaps=8)).cuda()
    _inject(0)
    try:
        with pytest.raises(sht.ShtError) as e:
            p.alm2map(a8)
        assert e.value.status == sht.SHT_ENOMEM
    finally:
        _inject(-1)
    assert torch.equal(p.alm2map(a8)[0:1], p.alm2map(a8[0:1]))
    # spin tables
    e2 = torch.zeros((1, 2, p.nalm), dtype=torch.complex128, device="cuda")
    _inject(0)
    try:
        with pytest.raises(sht.ShtError) as e:
            p.alm2map_spin(e2)
        assert e.value.status == sht.SHT_ENOMEM
    finally:
        _inject(-1)
    assert p.alm2map_spin(e2).abs().max().item() == 0.0
    p.close()
