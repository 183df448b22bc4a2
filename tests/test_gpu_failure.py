"""Failure detection on the GPU without a fault: a bounded device wait that runs out (an mbarrier
nobody arrives at) records SHT_ETIMEOUT in the plan's status word, the host reads it, and the
context stays usable for transforms afterwards."""
import ctypes

import numpy as np
import pytest

from paper_1106_0159_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_1106_0159_gb300 import sht
    p = sht.Plan(sht.healpix_geometry(64), 128, 128, grid=sht.GRID_HEALPIX)
    a = torch.from_numpy(inputs.gaussian_alm(128, 128, seed=91, nmaps=2)).cuda()
    before = p.alm2map(a).clone()
    assert p.device_status() == 0
    p.selftest_timeout()
    v = ctypes.c_int()
    assert sht.load().sht_plan_device_status(p._h, ctypes.byref(v), 0) == sht.SHT_ETIMEOUT and v.value & 1
    assert p.device_status(clear=True) & 1          # read and cleared
    assert p.device_status() == 0
    assert torch.equal(p.alm2map(a), before)         # the context still runs transforms
    p.set_mode(sht.MODE_SPLIT_BF16)
    assert p.map2alm(before).shape == (2, p.nalm) and p.device_status() == 0


def test_status_read_waits_for_work_on_a_nonblocking_stream():
    """The status read synchronises the whole device: a timeout recorded by a kernel still running
    on a non-blocking stream (torch's pool streams are) is seen without a manual synchronize."""
    from paper_1106_0159_gb300 import sht
    p = sht.Plan(sht.healpix_geometry(16), 32, 32, grid=sht.GRID_HEALPIX)
    assert p.device_status() == 0
    side = torch.cuda.Stream()
    p.selftest_timeout(stream=side)
    assert p.device_status(clear=True) & 1
    assert p.device_status() == 0
    p.close()
