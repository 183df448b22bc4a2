"""The C ABI library builds, loads and exports every symbol of include/sht.h;
its pure-host helpers and argument checks behave as documented (no GPU needed)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import geometry
from paper_1106_0159_gb300 import sht

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "sht.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sht_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    lib = sht.load()
    declared = _header_functions()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sht.EXPORTS) == declared


def test_nalm_and_index():
    for L, M in [(0, 0), (5, 5), (64, 64), (100, 37), (4096, 4096)]:
        assert sht.nalm(L, M) == (M + 1) * (L + 1) - M * (M + 1) // 2
        k = 0
        if L <= 100:
            for m in range(M + 1):
                for l in range(m, L + 1):
                    assert sht.alm_index(L, l, m) == k
                    k += 1
    lib = sht.load()
    assert lib.sht_nalm(3, 4) == -1
    assert lib.sht_alm_index(5, 2, 3) == -1


@pytest.mark.parametrize("nside", [1, 2, 16, 1024])
def test_healpix_helper_matches_oracle_geometry(nside):
    a = sht.healpix_geometry(nside)
    b = geometry.healpix(nside)
    assert np.array_equal(a[0], b[0])
    assert np.all(np.abs(a[1] - b[1]) <= np.spacing(b[1]))   # within one ulp
    assert np.max(np.abs(a[2] - b[2])) == 0.0
    assert np.max(np.abs(a[3] - b[3])) < 1e-30


@pytest.mark.parametrize("n", [1, 2, 5, 33, 2049])
def test_gauss_legendre_helper_matches_scipy(n):
    a = sht.gauss_legendre_geometry(n, 2 * n + 1)
    b = geometry.gauss_legendre(n, 2 * n + 1)
    assert np.array_equal(a[0], b[0])
    assert np.max(np.abs(np.cos(a[1]) - np.cos(b[1]))) < 2e-15
    # the helper works in double, with Newton's method in theta and Reinsch's difference form of
    # the Legendre recurrence near the poles; the oracle's nodes are polished in long double
    assert np.max(np.abs(a[1] - b[1]) / b[1]) < 1e-13
    assert np.max(np.abs(a[3] - b[3]) / b[3]) < 2e-12
    assert np.allclose(a[1] + a[1][::-1], math.pi, atol=1e-15, rtol=0)
    # what the transforms need: exact quadrature of P_l for l < 2n
    sp = pytest.importorskip("scipy.special")
    wg = a[3] * a[0] / (2 * math.pi)
    x = np.cos(a[1])
    # (the double-precision recurrence behind each weight carries up to ~3e-13 relative error at
    # n = 2049, ~1e-14 in the sum)
    for l in sorted(l for l in {0, 1, 2, n, 2 * n - 1} if l < 2 * n):
        exact = 2.0 if l == 0 else 0.0
        assert abs(float(np.sum(wg * sp.eval_legendre(l, x))) - exact) < 3e-14


def _create(nphi, theta, phi0, w, lmax, mmax):
    lib = sht.load()
    h = ctypes.c_void_p()
    arrs = [np.ascontiguousarray(nphi, np.int64)] + [np.ascontiguousarray(x, np.float64) for x in (theta, phi0, w)]
    st = lib.sht_plan_create(ctypes.byref(h), 0, len(arrs[0]), *[sht._np_ptr(a) for a in arrs], lmax, mmax)
    return st, h


def test_plan_create_rejects_bad_arguments_before_device_work():
    g = geometry.healpix(2)
    nphi, th, p0, w = [np.array(x) for x in g]
    cases = []
    cases.append((nphi, th, p0, w, 4, 5))               # mmax > lmax
    cases.append((nphi, th, p0, w, -1, 0))              # negative lmax
    bad = th.copy(); bad[0] = -0.1
    cases.append((nphi, bad, p0, w, 4, 4))              # theta < 0
    bad = th.copy(); bad[3] = math.pi + 1e-9
    cases.append((nphi, bad, p0, w, 4, 4))              # theta > pi
    badw = w.copy(); badw[2] = float("nan")
    cases.append((nphi, th, p0, badw, 4, 4))            # NaN weight
    badn = nphi.copy(); badn[1] = 0
    cases.append((badn, th, p0, w, 4, 4))               # empty ring
    for c in cases:
        st, h = _create(*c)
        assert st == sht.SHT_EINVAL
        assert not h.value
    lib = sht.load()
    h = ctypes.c_void_p()
    assert lib.sht_plan_create(ctypes.byref(h), 0, 0, None, None, None, None, 4, 4) == sht.SHT_EINVAL
    assert lib.sht_plan_create(None, 0, 1, None, None, None, None, 4, 4) == sht.SHT_EINVAL
    assert lib.sht_alm2map(None, None, None, 1, None) == sht.SHT_EINVAL
    assert lib.sht_plan_reserve(None, 1) == sht.SHT_EINVAL
    assert lib.sht_plan_set_tuning(None, 0, 4) == sht.SHT_EINVAL
    assert lib.sht_plan_tuning(None, 0) == -1
    assert lib.sht_plan_selftest_timeout(None, None) == sht.SHT_EINVAL
    assert lib.sht_alm2map_ws(None, None, None, 1, None, None, 0) == sht.SHT_EINVAL
    assert lib.sht_map2alm_ws(None, None, None, 1, None, None, 0) == sht.SHT_EINVAL
    assert lib.sht_alm2map_spin(None, 2, None, None, 1, None) == sht.SHT_EINVAL
    assert lib.sht_map2alm_spin(None, 2, None, None, 1, None) == sht.SHT_EINVAL
    assert lib.sht_spin_workspace_bytes(None, 1) == 0
    lv, tot = ctypes.c_int64(), ctypes.c_int64()
    assert lib.sht_plan_live_steps(None, ctypes.byref(lv), ctypes.byref(tot)) == sht.SHT_EINVAL
    assert lib.sht_status_string(sht.SHT_EINVAL) == b"invalid argument"
    assert lib.sht_plan_last_error(None) == b""


def test_geometry_helpers_reject_bad_sizes():
    lib = sht.load()
    z = np.zeros(4)
    n = np.zeros(4, np.int64)
    assert lib.sht_geom_healpix(0, sht._np_ptr(n), sht._np_ptr(z), sht._np_ptr(z), sht._np_ptr(z)) == sht.SHT_EINVAL
    assert lib.sht_geom_gauss_legendre(0, 5, sht._np_ptr(n), sht._np_ptr(z), sht._np_ptr(z),
                                       sht._np_ptr(z)) == sht.SHT_EINVAL
