"""Pins for the oracle's whole transforms (synthesis, analysis, and the two
separable stages).

The checks come from outside the oracle: closed forms of single modes, the
spherical-harmonic addition theorem (a point source in harmonic space gives
(2l+1)/(4 pi) P_l(cos gamma) with scipy's Legendre polynomial), exactness of
Gauss-Legendre quadrature (brute-force orthonormality and round trip), the
adjoint relation between synthesis and analysis, the pixel-shift property of
phi0, and agreement of the pixel-by-pixel and separable forms.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import geometry
from paper_1106_0159_gb300 import inputs


def _pix_angles(geom):
    nphi, theta, phi0, w = geom
    th, ph = [], []
    for r in range(len(nphi)):
        j = np.arange(nphi[r])
        th.append(np.full(nphi[r], theta[r]))
        ph.append(phi0[r] + 2 * np.pi * j / nphi[r])
    return np.concatenate(th), np.concatenate(ph)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2))


def test_single_mode_imaginary_y11():
    # a_11 = i: s = 2 Re(i Y_11) = -2 sqrt(3/(8 pi)) sin(theta) sin(phi); fixes the sign of phi
    geom = geometry.healpix(4)
    L = 6
    alm = np.zeros(oracle.nalm(L, L), dtype=np.complex128)
    alm[oracle.alm_index(L, 1, 1)] = 1j
    th, ph = _pix_angles(geom)
    ref = -2 * math.sqrt(3 / (8 * math.pi)) * np.sin(th) * np.sin(ph)
    for f in (oracle.alm2map_exact, oracle.alm2map_rings):
        s = f(geom, alm, L, L)
        assert np.max(np.abs(s - ref)) < 1e-14


def test_single_mode_y32_real():
    # a_32 = 1: s = 2 lambda_32(cos theta) cos(2 phi), lambda_32 = sqrt(105/(32 pi)) sin^2 cos
    geom = geometry.healpix(4)
    L = 5
    alm = np.zeros(oracle.nalm(L, L), dtype=np.complex128)
    alm[oracle.alm_index(L, 3, 2)] = 1.0
    th, ph = _pix_angles(geom)
    ref = 2 * math.sqrt(105 / (32 * math.pi)) * np.sin(th) ** 2 * np.cos(th) * np.cos(2 * ph)
    for f in (oracle.alm2map_exact, oracle.alm2map_rings):
        assert np.max(np.abs(f(geom, alm, L, L) - ref)) < 1e-14


@pytest.mark.parametrize("ell", [0, 1, 5, 12])
def test_addition_theorem_point_source(ell):
    # a_lm = conj(Y_lm(n0)) for one l (all m): sum_m a_lm Y_lm(n) = (2l+1)/(4pi) P_l(n . n0)
    sp = pytest.importorskip("scipy.special")
    geom = geometry.healpix(8)
    L = 16
    th0, ph0 = 0.83, 2.1
    alm = np.zeros(oracle.nalm(L, L), dtype=np.complex128)
    for m in range(ell + 1):
        lam = oracle.lambda_lm(th0, L, m)[ell - m]
        alm[oracle.alm_index(L, ell, m)] = lam * np.exp(-1j * m * ph0)
    th, ph = _pix_angles(geom)
    cosg = np.cos(th) * math.cos(th0) + np.sin(th) * math.sin(th0) * np.cos(ph - ph0)
    ref = (2 * ell + 1) / (4 * math.pi) * sp.eval_legendre(ell, cosg)
    for f in (oracle.alm2map_exact, oracle.alm2map_rings):
        assert np.max(np.abs(f(geom, alm, L, L) - ref)) < 1e-13


def test_gauss_legendre_orthonormality_brute_force():
    # Sum_pixels w Y_lm conj(Y_l'm') = delta on a GL grid with N > lmax rings and nphi > 2 mmax:
    # analysis of every unit coefficient (real and imaginary) returns that coefficient.
    L = 4
    geom = geometry.gauss_legendre(L + 1, 2 * L + 1)
    n = oracle.nalm(L, L)
    for k in range(n):
        for unit in (1.0, 1j):
            l_of_k = [l for m in range(L + 1) for l in range(m, L + 1)]
            m_of_k = [m for m in range(L + 1) for l in range(m, L + 1)]
            if m_of_k[k] == 0 and unit == 1j:
                continue
            a = np.zeros(n, dtype=np.complex128)
            a[k] = unit
            s = oracle.alm2map_exact(geom, a, L, L)
            b = oracle.map2alm_exact(geom, s, L, L)
            assert np.max(np.abs(b - a)) < 1e-14, (l_of_k[k], m_of_k[k], unit)


def test_gauss_legendre_round_trip_lmax32():
    L = 32
    geom = geometry.gauss_legendre(L + 1, 2 * L + 1)
    a = inputs.gaussian_alm(L, L, seed=3)[0]
    s = oracle.alm2map_rings(geom, a, L, L)
    b = oracle.map2alm_rings(geom, s, L, L)
    # the nodes enter as double theta = arccos(x_j), which moves them by ~1e-16/sin(theta);
    # the round-trip bar for the transforms is 1e-12 of the RMS
    assert _rel(b, a) < 1e-12


def test_gauss_legendre_round_trip_mmax_below_lmax():
    L, M = 24, 9
    geom = geometry.gauss_legendre(L + 1, 2 * M + 1)
    a = inputs.uniform_alm(L, M, seed=4)[0]
    s = oracle.alm2map_rings(geom, a, L, M)
    b = oracle.map2alm_rings(geom, s, L, M)
    assert _rel(b, a) < 1e-12


def _dot_alm(x, a, lmax, mmax):
    l, m = inputs.lm_arrays(lmax, mmax)
    w = np.where(m == 0, 1.0, 2.0)
    return float(np.sum(w * (x * np.conj(a)).real))


@pytest.mark.parametrize("form", ["exact", "rings"])
def test_adjoint_identity_healpix(form):
    # sum_p w_p s_p [alm2map(a)]_p = <map2alm(s), a>, <x,a> = sum x_l0 a_l0 + 2 Re sum_{m>0} x conj(a)
    geom = geometry.healpix(8)
    L = 16
    a = inputs.gaussian_alm(L, L, seed=5)[0]
    s = inputs.white_map(geometry.npix(geom), seed=6)[0]
    if form == "exact":
        syn = oracle.alm2map_exact(geom, a, L, L)
        ana = oracle.map2alm_exact(geom, s, L, L)
    else:
        syn = oracle.alm2map_rings(geom, a, L, L)
        ana = oracle.map2alm_rings(geom, s, L, L)
    wpix = np.repeat(geom[3], geom[0])
    lhs = float(np.sum(wpix * s * syn))
    rhs = _dot_alm(ana, a, L, L)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_separable_equals_pixel_by_pixel_healpix():
    geom = geometry.healpix(8)
    L, M = 20, 17   # mmax > nphi/2 on the polar rings: the phi sums alias
    a = inputs.gaussian_alm(L, M, seed=7)[0]
    s1 = oracle.alm2map_exact(geom, a, L, M)
    s2 = oracle.alm2map_rings(geom, a, L, M)
    assert _rel(s2, s1) < 1e-14
    s = inputs.white_map(geometry.npix(geom), seed=8)[0]
    b1 = oracle.map2alm_exact(geom, s, L, M)
    b2 = oracle.map2alm_rings(geom, s, L, M)
    assert _rel(b2, b1) < 1e-14


def test_constant_map_monopole():
    # equal-area HEALPix weights: a_00 of s = 1 is sum_p (4pi/npix) / sqrt(4pi) = sqrt(4 pi)
    geom = geometry.healpix(4)
    s = np.ones(geometry.npix(geom))
    a = oracle.map2alm_exact(geom, s, 8, 8)
    assert a[0].real == pytest.approx(math.sqrt(4 * math.pi), rel=1e-14)
    # and the monopole alone synthesises a constant 1/sqrt(4 pi)
    e = np.zeros(oracle.nalm(8, 8), dtype=np.complex128)
    e[0] = 1.0
    assert np.allclose(oracle.alm2map_exact(geom, e, 8, 8), 1 / math.sqrt(4 * math.pi), rtol=0, atol=1e-15)


def test_phi0_shift_rolls_ring():
    # moving phi0 by one pixel step rolls the ring by one pixel (reading of eq. Delta2map)
    geom = geometry.healpix(4)
    L = 10
    a = inputs.gaussian_alm(L, L, seed=9)[0]
    nphi, theta, phi0, w = geom
    r = 5
    d = oracle.delta_synth(geom, a, L, L, [r])
    base = oracle.ring_synth(geom, d, L, [r])
    phi0b = phi0.copy()
    phi0b[r] += 2 * np.pi / nphi[r]
    shifted = oracle.ring_synth((nphi, theta, phi0b, w), d, L, [r])
    assert np.max(np.abs(shifted - np.roll(base, -1))) < 1e-13


def test_stage_outputs_compose():
    # the Delta stages reproduce the composed transforms; Delta_0 and a_l0 are real
    geom = geometry.healpix(4)
    L = 12
    a = inputs.gaussian_alm(L, L, seed=10)[0]
    d = oracle.delta_synth(geom, a, L, L)
    assert np.all(d[:, 0].imag == 0)
    s = oracle.ring_synth(geom, d, L)
    assert _rel(s, oracle.alm2map_exact(geom, a, L, L)) < 1e-14
    ms = np.arange(L + 1)
    ds = oracle.delta_anal(geom, s, ms)
    b = np.concatenate(oracle.legendre_anal(geom, ds, L, ms))
    l, m = inputs.lm_arrays(L, L)
    assert np.all(b[m == 0].imag == 0)
    assert _rel(b, oracle.map2alm_exact(geom, s, L, L)) < 1e-14
