"""Pins for the oracle's ring geometries (HEALPix and Gauss-Legendre)."""
import math
import os

import numpy as np
import pytest

from oracle import geometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "healpix_rings_nside1_2.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            nside, i, nphi, zn, zd, p0 = line.split()
            rows.append((int(nside), int(i), int(nphi), int(zn) / int(zd), float(p0)))
    return rows


def test_healpix_small_tables_against_golden():
    rows = _golden_rows()
    for nside in (1, 2):
        nphi, theta, phi0, w = geometry.healpix(nside)
        mine = [r for r in rows if r[0] == nside]
        assert len(mine) == len(nphi) == 4 * nside - 1
        for (_, i, n, z, p0) in mine:
            assert nphi[i - 1] == n
            assert math.cos(theta[i - 1]) == pytest.approx(z, abs=1e-15)
            assert phi0[i - 1] == pytest.approx(p0 * math.pi, abs=1e-15)
        assert np.allclose(w, 4 * math.pi / (12 * nside * nside))


@pytest.mark.parametrize("nside", [1, 3, 8, 32, 1024])
def test_healpix_invariants(nside):
    nphi, theta, phi0, w = geometry.healpix(nside)
    assert len(nphi) == 4 * nside - 1
    assert int(nphi.sum()) == 12 * nside * nside
    # north/south mirror
    assert np.allclose(theta + theta[::-1], math.pi, atol=4e-15, rtol=0)
    assert np.all(nphi == nphi[::-1])
    # z continuous at the cap/belt boundary: cap formula at i = Nside gives 2/3
    assert math.cos(theta[nside - 1]) == pytest.approx(2.0 / 3.0, abs=1e-15)
    assert np.all(np.diff(theta) > 0)
    # equal-area weights integrate the constant exactly
    assert float(np.sum(w * nphi)) == pytest.approx(4 * math.pi, rel=1e-14)


def test_gauss_legendre_nodes_and_weights():
    sp = pytest.importorskip("scipy.special")
    N = 33
    nphi, theta, phi0, w = geometry.gauss_legendre(N, 65)
    x = np.cos(theta)
    xr, wr = sp.roots_legendre(N)
    assert np.allclose(np.sort(x), np.sort(xr), atol=1e-15, rtol=0)
    assert np.all(np.diff(theta) > 0)          # north first
    wg = w * nphi / (2 * math.pi)
    assert float(wg.sum()) == pytest.approx(2.0, rel=1e-14)
    # exact for polynomials of degree < 2N
    for k in range(0, 2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert float(np.sum(wg * x ** k)) == pytest.approx(exact, abs=1e-14)
    assert np.all(phi0 == 0)
