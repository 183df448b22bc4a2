"""Pins for the oracle's normalised associated Legendre functions lambda_lm.

Each check ties the oracle to something other than itself: closed forms of
low-degree harmonics, exact rational arithmetic for mu_m (eq. pmm), the
Unsold sum rule, the Bonnet recurrence for Legendre polynomials, scipy's
spherical harmonics, and the parity and pole values of the functions.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

THETAS = [1e-3, 0.05, 0.3, 0.7, 1.2, math.pi / 2, 2.0, math.pi - 0.01]


def test_closed_forms_low_degree():
    # Y_00, Y_10, Y_20, Y_11, Y_21, Y_22 without the Condon-Shortley phase (lambda_mm > 0)
    for th in THETAS:
        x, s = math.cos(th), math.sin(th)
        l0 = oracle.lambda_lm(th, 3, 0)
        assert l0[0] == pytest.approx(1 / math.sqrt(4 * math.pi), rel=1e-15)
        assert l0[1] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * x, rel=1e-14, abs=1e-17)
        assert l0[2] == pytest.approx(math.sqrt(5 / (4 * math.pi)) * (3 * x * x - 1) / 2, rel=1e-13, abs=1e-16)
        l1 = oracle.lambda_lm(th, 2, 1)
        assert l1[0] == pytest.approx(math.sqrt(3 / (8 * math.pi)) * s, rel=1e-14)
        assert l1[1] == pytest.approx(math.sqrt(15 / (8 * math.pi)) * s * x, rel=1e-13, abs=1e-17)
        l2 = oracle.lambda_lm(th, 2, 2)
        assert l2[0] == pytest.approx(math.sqrt(15 / (32 * math.pi)) * s * s, rel=1e-14)


def _mu_exact(m: int) -> Fraction:
    # mu_m^2 = (2m+1)! / (4 pi 4^m (m!)^2), without the 1/(4 pi): prod_{k=1..m} (2k+1)/(2k)
    f = Fraction(1)
    for k in range(1, m + 1):
        f *= Fraction(2 * k + 1, 2 * k)
    return f


@pytest.mark.parametrize("m", [0, 1, 2, 5, 17, 64, 150, 300])
def test_log_mu_against_exact_rational(m):
    exact = 0.5 * (math.log(_mu_exact(m)) - math.log(4 * math.pi))
    assert oracle.log_mu(m) == pytest.approx(exact, abs=1e-13)


@pytest.mark.parametrize("m", [1, 3, 10, 40, 100, 250])
def test_sectoral_lambda_mm(m):
    # lambda_mm = mu_m sin^m(theta), eq. (pmm)
    for th in [0.4, 1.0, math.pi / 2, 2.5]:
        mu = math.sqrt(float(_mu_exact(m)) / (4 * math.pi))
        expect = mu * math.sin(th) ** m
        got = oracle.lambda_lm(th, m, m)[0]
        assert got == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("th", [1e-3, 0.02, 0.3, 1.0, math.pi / 2, math.pi - 0.3])
def test_unsold_sum_rule_high_degree(th):
    # sum_m |Y_lm|^2 = lambda_l0^2 + 2 sum_{m>0} lambda_lm^2 = (2l+1)/(4 pi), every l <= 2048
    L = 2048
    tot = np.zeros(L + 1)
    for m in range(L + 1):
        c = oracle.lambda_lm(th, L, m)
        tot[m:] += (1.0 if m == 0 else 2.0) * c * c
    ratio = tot * 4 * np.pi / (2 * np.arange(L + 1) + 1)
    assert np.max(np.abs(ratio - 1)) < 1e-13


def test_unsold_sum_rule_lmax_4096():
    L = 4096
    for th in [0.01, 1.1]:
        tot = np.zeros(L + 1)
        for m in range(L + 1):
            c = oracle.lambda_lm(th, L, m)
            tot[m:] += (1.0 if m == 0 else 2.0) * c * c
        ratio = tot * 4 * np.pi / (2 * np.arange(L + 1) + 1)
        assert np.max(np.abs(ratio - 1)) < 1e-13


def test_lambda_l0_against_bonnet():
    # lambda_l0 = sqrt((2l+1)/(4 pi)) P_l(x), P_l from (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}
    # Evaluated in numpy long double: near the poles P_l'(x) ~ l^2/2, so cos(theta) rounded to
    # double would already move P_l by ~l^2 * 1e-16.
    L = 1000
    ld = np.longdouble
    for th in THETAS:
        x = np.cos(ld(th))
        p = np.zeros(L + 1, dtype=ld)
        p[0] = ld(1)
        p[1] = x
        for l in range(1, L):
            p[l + 1] = ((2 * l + 1) * x * p[l] - l * p[l - 1]) / (l + 1)
        ref = (np.sqrt((2 * np.arange(L + 1, dtype=ld) + 1) / (4 * ld(np.pi))) * p).astype(np.float64)
        got = oracle.lambda_lm(th, L, 0)
        scale = np.sqrt((2 * np.arange(L + 1) + 1) / (4 * np.pi))
        assert np.max(np.abs(got - ref) / scale) < 1e-14


def test_against_scipy_spherical_harmonics():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    L = 60
    for th in THETAS:
        for m in range(0, L + 1, 7):
            got = oracle.lambda_lm(th, L, m)
            ls = np.arange(m, L + 1)
            ref = np.array([sp.sph_harm_y(int(l), m, th, 0.0).real for l in ls]) * (-1.0) ** m
            scale = np.sqrt((2 * ls + 1) / (4 * np.pi))
            assert np.max(np.abs(got - ref) / scale) < 1e-12, (th, m)


def test_parity_and_poles():
    L = 300
    for th in [0.1, 0.6, 1.3]:
        for m in [0, 1, 7, 50, 200]:
            a = oracle.lambda_lm(th, L, m)
            b = oracle.lambda_lm(math.pi - th, L, m)
            sign = (-1.0) ** (np.arange(m, L + 1) + m)
            assert np.max(np.abs(b - sign * a)) < 1e-12 * max(1.0, np.max(np.abs(a)))
    top = oracle.lambda_lm(0.0, L, 0)
    assert np.allclose(top, np.sqrt((2 * np.arange(L + 1) + 1) / (4 * np.pi)), rtol=1e-13)
    for m in [1, 2, 30]:
        assert np.all(oracle.lambda_lm(0.0, L, m) == 0.0)
        # sin(double(pi)) ~ 1.2e-16, so only approximately zero at the south pole
        assert np.max(np.abs(oracle.lambda_lm(math.pi, L, m))) < 1e-9


def test_deep_underflow_start_is_zero_not_nan():
    # near the pole with large m the start value lies far below the double range
    c = oracle.lambda_lm(1e-4, 4096, 3000)
    assert np.all(np.isfinite(c))
    assert np.all(c == 0.0)
