"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no transform arithmetic: it only draws random numbers in
the layouts the library uses.

* ``gaussian_alm``: CMB-like coefficients, a_l0 ~ N(0, C_l) real and, for
  m > 0, Re and Im ~ N(0, C_l / 2), with C_l = 1 / (l (l + 1) + 1).
* ``uniform_alm``: Re and Im uniform in (-1, 1), a_l0 real -- the input of
  the paper's accuracy experiments (Section 5, eq. error).
* ``white_map``: unit-variance Gaussian pixels.

Coefficients are complex128 in m-major triangular order,
index(l, m) = m (2 lmax + 3 - m) / 2 + (l - m).
"""
from __future__ import annotations

import numpy as np


def nalm(lmax: int, mmax: int) -> int:
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def lm_arrays(lmax: int, mmax: int):
    """(l, m) of every coefficient in m-major order."""
    ls, ms = [], []
    for m in range(mmax + 1):
        ls.append(np.arange(m, lmax + 1, dtype=np.int64))
        ms.append(np.full(lmax - m + 1, m, dtype=np.int64))
    return np.concatenate(ls), np.concatenate(ms)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_alm(lmax: int, mmax: int, seed: int, nmaps: int = 1) -> np.ndarray:
    """[nmaps][nalm] complex128 with variance C_l = 1 / (l (l + 1) + 1)."""
    g = _rng(seed)
    l, m = lm_arrays(lmax, mmax)
    cl = 1.0 / (l * (l + 1.0) + 1.0)
    n = l.size
    re = g.standard_normal((nmaps, n))
    im = g.standard_normal((nmaps, n))
    sd = np.where(m == 0, np.sqrt(cl), np.sqrt(cl / 2.0))
    a = (re * sd) + 1j * (im * sd)
    a[:, m == 0] = a[:, m == 0].real
    return np.ascontiguousarray(a)


def uniform_alm(lmax: int, mmax: int, seed: int, nmaps: int = 1) -> np.ndarray:
    """[nmaps][nalm] complex128, Re and Im uniform in (-1, 1), a_l0 real."""
    g = _rng(seed)
    l, m = lm_arrays(lmax, mmax)
    n = l.size
    a = g.uniform(-1.0, 1.0, (nmaps, n)) + 1j * g.uniform(-1.0, 1.0, (nmaps, n))
    a[:, m == 0] = a[:, m == 0].real
    return np.ascontiguousarray(a)


def white_map(npix: int, seed: int, nmaps: int = 1) -> np.ndarray:
    """[nmaps][npix] float64, unit-variance Gaussian."""
    return np.ascontiguousarray(_rng(seed).standard_normal((nmaps, int(npix))))


def random_delta(nrings: int, mmax: int, seed: int, nmaps: int = 1) -> np.ndarray:
    """[nmaps][nrings][mmax+1] complex128 unit Gaussian, Delta_0 real (ring-stage tests)."""
    g = _rng(seed)
    d = g.standard_normal((nmaps, nrings, mmax + 1)) + 1j * g.standard_normal((nmaps, nrings, mmax + 1))
    d[:, :, 0] = d[:, :, 0].real
    return np.ascontiguousarray(d)
