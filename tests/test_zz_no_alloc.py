"""sht_alm2map_noalloc: the synthesis entry point for callers that cannot
allocate device memory during a transform (code running inside another
framework's memory pool or under a fixed memory budget, or that must avoid
the device synchronisation an allocation can cause).  Its scratch is a static
device array, so the call itself allocates nothing.  Its output must agree
with sht_alm2map's, on two calls in a row (the second reuses the array the
first one left behind), and it runs the plan's own arithmetic (FP64 or the
precision form).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(x, ref):
    return float(np.max(np.abs(x - ref)) / np.sqrt(np.mean(ref ** 2)))


def _call(lib, plan, a, out):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.sht_alm2map_noalloc(plan._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   int(a.shape[0]), s)


def test_noalloc_matches_alm2map_on_two_calls_in_a_row():
    from paper_1106_0159_gb300 import sht
    lib = sht.load()
    L = 64
    plan = sht.Plan(sht.healpix_geometry(32), L, L, grid=sht.GRID_HEALPIX)
    outs = []
    for seed in (41, 42):
        a = torch.from_numpy(inputs.gaussian_alm(L, L, seed=seed, nmaps=3)).cuda()
        ref = plan.alm2map(a)
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert _call(lib, plan, a, out) == sht.SHT_OK, lib.sht_plan_last_error(plan._h)
        torch.cuda.synchronize()
        if outs:  # the scratch array exists already: the call must not take device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, want) <= TOL
        outs.append(got)
    assert not np.array_equal(outs[0], outs[1])
    plan.close()


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_noalloc_runs_the_plan_mode_and_matches_the_oracle(mode):
    """HEALPix Nside 32, lmax 64, one map (the smallest benchmark configuration): the no-alloc
    synthesis takes the plan's own arithmetic, so on a precision-form plan it gives exactly what
    sht_alm2map gives there, and in either mode it matches the oracle's pixel-by-pixel synthesis
    within that mode's tolerance (1e-11 FP64, 1e-9 precision form)."""
    import oracle
    from oracle import geometry
    from paper_1106_0159_gb300 import sht
    lib = sht.load()
    L, nside = 64, 32
    geom = geometry.healpix(nside)
    plan = sht.Plan(geom, L, L, grid=sht.GRID_HEALPIX)
    if mode == "split":
        plan.set_mode(sht.MODE_SPLIT_BF16)
    a_h = inputs.gaussian_alm(L, L, seed=43, nmaps=1)
    a = torch.from_numpy(a_h).cuda()
    ref = plan.alm2map(a)
    out = torch.full_like(ref, float("nan"))
    for _ in range(2):
        assert _call(lib, plan, a, out) == sht.SHT_OK, lib.sht_plan_last_error(plan._h)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    want = oracle.alm2map_exact(geom, a_h[0], L, L)
    assert _rel(out.cpu().numpy()[0], want) <= (TOL if mode == "fp64" else 1e-9)
    plan.close()


def test_noalloc_rejects_work_beyond_the_static_scratch():
    from paper_1106_0159_gb300 import sht
    lib = sht.load()
    cap = int(lib.sht_noalloc_scratch_bytes())
    assert cap == 64 << 20
    plan = sht.Plan(sht.healpix_geometry(1024), 2048)   # Delta alone needs 4095 * 2049 * 16 B > 64 MiB
    a = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, plan.npix), dtype=torch.float64, device="cuda")
    assert _call(lib, plan, a, out) == sht.SHT_EINVAL
    assert b"static scratch" in lib.sht_plan_last_error(plan._h)
    with pytest.raises(ValueError):
        plan.alm2map_noalloc(a, out=out)
    plan.close()
