"""Pins of the spin-2 oracle (oracle/spin_oracle.c) to things other than itself: the explicit
spin-weighted harmonic sum of Goldberg et al. (1967) evaluated in 50-digit arithmetic, closed
forms of the l = 2 functions, the spin sum rule, the reflection symmetry, the scalar oracle at
s = 0, and exact Gauss-Legendre quadrature (the round trip is the identity)."""
import math

import numpy as np
import pytest

import oracle
from oracle import geometry
from paper_1106_0159_gb300 import inputs


def goldberg(l, m, s, theta, mp):
    """slambda_lm from the explicit finite sum (no Condon-Shortley factor), in mpmath."""
    if l < max(abs(m), abs(s)):
        return mp.mpf(0)
    th = mp.mpf(theta)
    sh, ch = mp.sin(th / 2), mp.cos(th / 2)
    f = mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * (2 * l + 1) /
                (4 * mp.pi * mp.factorial(l + s) * mp.factorial(l - s)))
    tot = mp.mpf(0)
    for r in range(0, l - s + 1):
        k = r + s - m
        if k < 0 or k > l + s:
            continue
        tot += (mp.binomial(l - s, r) * mp.binomial(l + s, k) * (-1) ** (l - r - s) *
                sh ** (2 * l - 2 * r - s + m) * ch ** (2 * r + s - m))
    return f * tot


@pytest.mark.parametrize("theta", [0.01, 0.3, 1.1, math.pi / 2, 2.5, 3.1])
def test_spin_lambda_matches_the_explicit_sum(theta):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    L = 14
    worst = 0.0
    for s in (2, -2):
        for m in range(0, L + 1):
            got = oracle.spin_lambda(theta, L, m, s)
            want = np.array([float(goldberg(l, m, s, theta, mp)) for l in range(m, L + 1)])
            scale = max(np.max(np.abs(want)), 1e-300)
            worst = max(worst, float(np.max(np.abs(got - want)) / scale))
    assert worst < 1e-13


def test_spin_lambda_closed_forms_l2():
    for th in (0.0, 0.2, 1.0, 2.0, math.pi):
        sh2, ch2 = math.sin(th / 2) ** 2, math.cos(th / 2) ** 2
        # 2Y_22 = (1/8) sqrt(5/pi) (1 - cos)^2 e^{2 i phi}; (-2)Y_22 = (1/8) sqrt(5/pi) (1 + cos)^2 e^{2 i phi}
        assert oracle.spin_lambda(th, 2, 2, 2)[0] == pytest.approx(math.sqrt(5 / (4 * math.pi)) * sh2 ** 2, abs=1e-15)
        assert oracle.spin_lambda(th, 2, 2, -2)[0] == pytest.approx(math.sqrt(5 / (4 * math.pi)) * ch2 ** 2, abs=1e-15)
        # (+-2)Y_20 = (1/4) sqrt(15/(2 pi)) sin^2(theta)
        want = math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2
        assert oracle.spin_lambda(th, 2, 0, 2)[2] == pytest.approx(want, abs=1e-15)
        assert oracle.spin_lambda(th, 2, 0, -2)[2] == pytest.approx(want, abs=1e-15)
        # below l = 2 nothing exists
        assert np.all(oracle.spin_lambda(th, 2, 0, 2)[:2] == 0.0)
        assert oracle.spin_lambda(th, 2, 1, -2)[0] == 0.0


def test_spin_zero_is_the_scalar_oracle():
    for th in (1e-3, 0.4, 1.3, math.pi / 2, 2.9):
        for m in (0, 1, 7, 100, 511):
            a = oracle.spin_lambda(th, 512, m, 0)
            b = oracle.lambda_lm(th, 512, m)
            assert np.max(np.abs(a - b)) <= 1e-13 * max(np.max(np.abs(b)), 1e-300)


def _spin_sum(theta, L):
    tot = np.zeros(L + 1)
    for m in range(0, L + 1):
        p = oracle.spin_lambda(theta, L, m, 2)
        tot[m:] += p ** 2
        if m > 0:
            q = oracle.spin_lambda(theta, L, m, -2)
            tot[m:] += q ** 2
    return tot


@pytest.mark.parametrize("theta,L,tol", [(1e-3, 1024, 1e-13), (0.05, 1024, 1e-13), (0.9, 1024, 1e-13),
                                          (math.pi / 2, 1024, 1e-13), (3.0, 1024, 1e-13), (1.2, 4096, 1e-13),
                                          (2e-4, 4096, 1e-12)])
def test_spin_sum_rule(theta, L, tol):
    # sum over all m of |sY_lm|^2 = (2l+1)/(4 pi); negative m are the (-s) functions of |m|.
    # Next to a pole the l-recurrence is nearly degenerate and its rounding errors grow like
    # eps l^1.5 / sin(theta): with the 64-bit long double mantissa of x86 that is ~3e-13 at
    # theta = 2e-4, l = 4096 (binary128 on aarch64 is far below), hence the wider bound there.
    tot = _spin_sum(theta, L)
    l = np.arange(2, L + 1)
    want = (2 * l + 1) / (4 * math.pi)
    assert np.max(np.abs(tot[2:] - want) / want) < tol


def test_spin_reflection_symmetry():
    th = 0.83
    for m in (0, 1, 2, 5, 40):
        for s in (2, -2):
            a = oracle.spin_lambda(math.pi - th, 200, m, s)
            b = oracle.spin_lambda(th, 200, m, -s)
            sign = np.array([(-1) ** (l + m) for l in range(m, 201)])
            assert np.max(np.abs(a - sign * b)) <= 1e-13 * np.max(np.abs(b))


def _rand_eb(L, seed):
    E = inputs.uniform_alm(L, L, seed=seed)[0]
    B = inputs.uniform_alm(L, L, seed=seed + 1)[0]
    lv, _ = inputs.lm_arrays(L, L)
    E[lv < 2] = 0.0
    B[lv < 2] = 0.0
    return E, B


def test_exact_round_trip_on_gauss_legendre_is_identity():
    L = 8
    geom = geometry.gauss_legendre(L + 2, 2 * L + 4)
    E, B = _rand_eb(L, 11)
    q, u = oracle.spin_alm2map_exact(geom, E, B, L, L)
    E2, B2 = oracle.spin_map2alm_exact(geom, q, u, L, L)
    rms = np.sqrt(np.mean(np.abs(E) ** 2))
    assert np.max(np.abs(E2 - E)) / rms < 1e-13
    assert np.max(np.abs(B2 - B)) / rms < 1e-13


def test_separable_forms_equal_the_exact_ones():
    L = 10
    geom = geometry.healpix(4)
    E, B = _rand_eb(L, 21)
    q, u = oracle.spin_alm2map_exact(geom, E, B, L, L)
    q2, u2 = oracle.spin_alm2map_rings(geom, E, B, L, L)
    sc = np.sqrt(np.mean(q ** 2 + u ** 2))
    assert np.max(np.abs(q2 - q)) / sc < 1e-14 and np.max(np.abs(u2 - u)) / sc < 1e-14
    Ea, Ba = oracle.spin_map2alm_exact(geom, q, u, L, L)
    Eb, Bb = oracle.spin_map2alm_rings(geom, q, u, L, L)
    sc = np.sqrt(np.mean(np.abs(Ea) ** 2))
    assert np.max(np.abs(Eb - Ea)) / sc < 1e-14 and np.max(np.abs(Bb - Ba)) / sc < 1e-14


def test_separable_round_trip_gauss_legendre():
    L = 40
    geom = geometry.gauss_legendre(L + 1, 2 * L + 1)
    E, B = _rand_eb(L, 31)
    q, u = oracle.spin_alm2map_rings(geom, E, B, L, L)
    E2, B2 = oracle.spin_map2alm_rings(geom, q, u, L, L)
    rms = np.sqrt(np.mean(np.abs(E) ** 2))
    assert np.max(np.abs(E2 - E)) / rms < 1e-12 and np.max(np.abs(B2 - B)) / rms < 1e-12


def test_single_axisymmetric_modes():
    # E_l0 = 1 alone: U = 0 and Q = -2lambda_l0(theta) (W = 2lambda = (-2)lambda, X = 0 at m = 0);
    # B_l0 = 1 alone: Q = 0 and U = -2lambda_l0
    L, l = 6, 4
    geom = geometry.healpix(2)
    nphi, theta = geom[0], geom[1]
    E = np.zeros(oracle.nalm(L, L), dtype=np.complex128)
    B = np.zeros_like(E)
    E[oracle.alm_index(L, l, 0)] = 1.0
    q, u = oracle.spin_alm2map_exact(geom, E, B, L, L)
    want = np.concatenate([np.full(int(n), -oracle.spin_lambda(t, L, 0, 2)[l]) for n, t in zip(nphi, theta)])
    assert np.max(np.abs(u)) < 1e-15 and np.max(np.abs(q - want)) < 1e-15
    q, u = oracle.spin_alm2map_exact(geom, B, E, L, L)
    assert np.max(np.abs(q)) < 1e-15 and np.max(np.abs(u - want)) < 1e-15


def test_phi_rotation_of_a_single_mode():
    # E_lm = 1 (m > 0): Q + iU picks up exp(i m dphi) under a rotation about the axis, which a
    # shift of every ring's phi0 by dphi realises
    L, l, m, dphi = 6, 5, 3, 0.37
    geom = geometry.healpix(2)
    nphi, theta, phi0, w = geom
    E = np.zeros(oracle.nalm(L, L), dtype=np.complex128)
    B = np.zeros_like(E)
    E[oracle.alm_index(L, l, m)] = 1.0
    q, u = oracle.spin_alm2map_exact(geom, E, B, L, L)
    E2 = E.copy()
    E2[oracle.alm_index(L, l, m)] = np.exp(1j * m * dphi)
    q2, u2 = oracle.spin_alm2map_exact((nphi, theta, np.asarray(phi0) - dphi, w), E2, B, L, L)
    assert np.max(np.abs(q2 - q)) < 1e-14 and np.max(np.abs(u2 - u)) < 1e-14
