"""Ring geometries for the oracle (test infrastructure only).

Section 2.2 of the paper requires iso-latitude rings with equidistant pixels,
phi_j = phi0 + j * 2 pi / nphi.  Two grids are built here from their
published definitions:

* HEALPix (Gorski et al. 2005, cited in Section 2.2): rings i = 1..4 Nside - 1
  from north to south; polar cap i < Nside has nphi = 4 i,
  z = 1 - i^2 / (3 Nside^2), phi0 = pi / (4 i); the equatorial belt
  Nside <= i <= 3 Nside has nphi = 4 Nside, z = 4/3 - 2 i / (3 Nside),
  phi0 = pi / (4 Nside) when i - Nside is even and 0 otherwise; the south
  cap mirrors the north one with z -> -z.  Pixels are equal-area, so the
  quadrature weight of every pixel is 4 pi / npix.
* Gauss-Legendre: the N roots x_j of P_N (scipy, Newton-polished), north first, equal nphi,
  phi0 = 0, per-pixel weight 2 pi w_j / nphi with w_j the Gauss weights.

Each builder returns (nphi int64[R], theta float64[R], phi0 float64[R],
w float64[R]).
"""
from __future__ import annotations

import numpy as np


def healpix(nside: int):
    nside = int(nside)
    nr = 4 * nside - 1
    npix = 12 * nside * nside
    nphi = np.zeros(nr, dtype=np.int64)
    theta = np.zeros(nr, dtype=np.float64)
    phi0 = np.zeros(nr, dtype=np.float64)
    for k in range(nr):
        i = k + 1
        north = i if i <= 2 * nside else 4 * nside - i
        if north < nside:
            n = 4 * north
            # 1 - z = north^2 / (3 Nside^2); theta = 2 asin(sqrt((1 - z) / 2)) keeps the
            # polar rings accurate.
            th = 2.0 * np.arcsin(north / (np.sqrt(6.0) * nside))
            p0 = np.pi / (4.0 * north)
        else:
            n = 4 * nside
            z = 4.0 / 3.0 - 2.0 * north / (3.0 * nside)
            th = np.arccos(z)
            p0 = np.pi / (4.0 * nside) if ((i - nside) % 2 == 0) else 0.0
        if i > 2 * nside:
            th = np.pi - th
        nphi[k] = n
        theta[k] = th
        phi0[k] = p0
    assert int(nphi.sum()) == npix
    w = np.full(nr, 4.0 * np.pi / npix, dtype=np.float64)
    return nphi, theta, phi0, w


def _legendre_and_derivative(x, n):
    """P_n(x) and P_n'(x) by the Bonnet recurrence, in x's dtype."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    for l in range(2, n + 1):
        p0, p1 = p1, ((2 * l - 1) * x * p1 - (l - 1) * p0) / l
    if n == 0:
        return p0, np.zeros_like(x)
    dp = n * (x * p1 - p0) / (x * x - 1)
    return p1, dp


def gauss_legendre(nrings: int, nphi: int):
    from scipy.special import roots_legendre

    n = int(nrings)
    x0, _ = roots_legendre(n)
    # scipy's nodes, polished by two Newton steps in long double (scipy's weights for
    # n in the thousands are only good to ~1e-13); weights 2 / ((1 - x^2) P_n'(x)^2)
    x = x0.astype(np.longdouble)
    for _ in range(2):
        p, dp = _legendre_and_derivative(x, n)
        x = x - p / dp
    _, dp = _legendre_and_derivative(x, n)
    wg = 2 / ((1 - x * x) * dp * dp)
    order = np.argsort(-x)  # north (x = cos theta near +1) first
    x = x[order]
    wg = wg[order].astype(np.float64)
    theta = np.arccos(x).astype(np.float64)
    nphi_a = np.full(int(nrings), int(nphi), dtype=np.int64)
    phi0 = np.zeros(int(nrings), dtype=np.float64)
    w = 2.0 * np.pi * wg / float(nphi)
    return nphi_a, theta, phi0, w


def npix(geom) -> int:
    return int(np.asarray(geom[0]).sum())


def ring_offsets(geom) -> np.ndarray:
    n = np.asarray(geom[0], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(n)])
