"""Oracle for the spherical harmonic transforms of arXiv:1106.0159.

TEST INFRASTRUCTURE ONLY: a plain, slow CPU statement of what the
transforms compute (long double C in ``sht_oracle.c`` plus the numpy
geometry in ``geometry.py``).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never
does, and the two share no code.

Every function takes the ring geometry as four per-ring arrays
(``nphi``, ``theta``, ``phi0``, ``w``) and complex coefficients in the
m-major triangular layout ``index(l, m) = m (2 lmax + 3 - m) / 2 + (l - m)``.

Parity pins (what each part is checked against) live in
``tests/test_oracle_*.py``; nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import geometry  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_SPIN_SRC = os.path.join(_HERE, "spin_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``sht_oracle.c`` and ``spin_oracle.c`` into ``liboracle.so`` with gcc (OpenMP, -O2,
    no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SPIN_SRC))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, _SPIN_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        sigs = {
            "oracle_lambda": [D, I, I, P],
            "oracle_delta_synth": [I, P, I, I, P, I, P, P],
            "oracle_ring_synth": [I, P, P, I, I, P, P, P],
            "oracle_alm2map_exact": [I, P, P, P, I, I, P, P],
            "oracle_map2alm_exact": [I, P, P, P, P, I, I, P, P],
            "oracle_delta_anal": [I, P, P, P, P, I, P, P],
            "oracle_legendre_anal": [I, P, I, I, P, P, P],
            "oracle_spin_lambda": [D, I, I, I, P],
            "oracle_spin_delta_synth": [I, P, I, I, P, P, I, P, P, P],
            "oracle_spin_legendre_anal": [I, P, I, I, P, P, P, P, P],
            "oracle_spin_alm2map_exact": [I, P, P, P, I, I, P, P, P, P],
            "oracle_spin_map2alm_exact": [I, P, P, P, P, I, I, P, P, P, P],
        }
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = None
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_set_threads.restype = I
        lib.oracle_log_mu.argtypes = [I]
        lib.oracle_log_mu.restype = D
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def nalm(lmax: int, mmax: int) -> int:
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def alm_index(lmax: int, l: int, m: int) -> int:
    return m * (2 * lmax + 3 - m) // 2 + (l - m)


def set_threads(n: int) -> int:
    """Host threads of the oracle's parallel loops from now on (timing only; results do not
    depend on it).  Returns the previous count."""
    return int(_load().oracle_set_threads(int(n)))


def lambda_lm(theta: float, lmax: int, m: int) -> np.ndarray:
    """lambda_{l m}(cos theta) for l = m..lmax (Section 2.1, eqs. assLegRec/pmm/pm1m)."""
    out = np.zeros(lmax - m + 1, dtype=np.float64)
    _load().oracle_lambda(float(theta), int(lmax), int(m), _p(out))
    return out


def log_mu(m: int) -> float:
    """ln mu_m of eq. (pmm)."""
    return float(_load().oracle_log_mu(int(m)))


def delta_synth(geom, alm, lmax: int, mmax: int, rings=None) -> np.ndarray:
    """Delta^A_m(r) of eq. (DeltaDef), shape [len(rings)][mmax+1] complex."""
    nphi, theta, phi0, w = geom
    theta = _f64(theta)
    rings = _i32(np.arange(len(theta)) if rings is None else rings)
    alm = _c128(alm)
    assert alm.size == nalm(lmax, mmax)
    out = np.zeros((len(rings), mmax + 1), dtype=np.complex128)
    _load().oracle_delta_synth(len(theta), _p(theta), lmax, mmax, _p(alm), len(rings), _p(rings), _p(out))
    return out


def ring_synth(geom, delta, mmax: int, rings=None) -> np.ndarray:
    """Pixels of the selected rings from Delta^A (eq. Delta2map), concatenated."""
    nphi, theta, phi0, w = geom
    nphi = _i64(nphi)
    phi0 = _f64(phi0)
    rings = _i32(np.arange(len(nphi)) if rings is None else rings)
    delta = _c128(delta)
    assert delta.shape == (len(rings), mmax + 1)
    out = np.zeros(int(nphi[rings].sum()), dtype=np.float64)
    _load().oracle_ring_synth(len(nphi), _p(nphi), _p(phi0), mmax, len(rings), _p(rings), _p(delta), _p(out))
    return out


def alm2map_rings(geom, alm, lmax: int, mmax: int, rings=None) -> np.ndarray:
    """Separable synthesis (Section 2.2) of the selected rings."""
    rings = np.arange(len(geom[0])) if rings is None else np.asarray(rings)
    d = delta_synth(geom, alm, lmax, mmax, rings)
    return ring_synth(geom, d, mmax, rings)


def alm2map_exact(geom, alm, lmax: int, mmax: int) -> np.ndarray:
    """Pixel-by-pixel synthesis, eq. (alm2mapDef)."""
    nphi, theta, phi0, w = geom
    nphi, theta, phi0 = _i64(nphi), _f64(theta), _f64(phi0)
    alm = _c128(alm)
    assert alm.size == nalm(lmax, mmax)
    out = np.zeros(int(nphi.sum()), dtype=np.float64)
    _load().oracle_alm2map_exact(len(nphi), _p(nphi), _p(theta), _p(phi0), lmax, mmax, _p(alm), _p(out))
    return out


def map2alm_exact(geom, m_, lmax: int, mmax: int) -> np.ndarray:
    """Pixel-by-pixel analysis, eq. (map2almDef) with conj(Y)."""
    nphi, theta, phi0, w = geom
    nphi, theta, phi0, w = _i64(nphi), _f64(theta), _f64(phi0), _f64(w)
    m_ = _f64(m_)
    assert m_.size == nphi.sum()
    out = np.zeros(nalm(lmax, mmax), dtype=np.complex128)
    _load().oracle_map2alm_exact(len(nphi), _p(nphi), _p(theta), _p(phi0), _p(w), lmax, mmax, _p(m_), _p(out))
    return out


def delta_anal(geom, m_, ms) -> np.ndarray:
    """Delta^S_m(r) of eq. (almfftdef), shape [len(ms)][nrings] complex (weight included)."""
    nphi, theta, phi0, w = geom
    nphi, phi0, w = _i64(nphi), _f64(phi0), _f64(w)
    m_ = _f64(m_)
    ms = _i32(ms)
    out = np.zeros((len(ms), len(nphi)), dtype=np.complex128)
    _load().oracle_delta_anal(len(nphi), _p(nphi), _p(phi0), _p(w), _p(m_), len(ms), _p(ms), _p(out))
    return out


def legendre_anal(geom, delta, lmax: int, ms) -> list:
    """a_lm for l = m..lmax from Delta^S (eq. almdef); one array per selected m."""
    nphi, theta, phi0, w = geom
    theta = _f64(theta)
    ms = _i32(ms)
    delta = _c128(delta)
    assert delta.shape == (len(ms), len(theta))
    sizes = [lmax - int(m) + 1 for m in ms]
    out = np.zeros(sum(sizes), dtype=np.complex128)
    _load().oracle_legendre_anal(len(theta), _p(theta), lmax, len(ms), _p(ms), _p(delta), _p(out))
    res, o = [], 0
    for s in sizes:
        res.append(out[o:o + s].copy())
        o += s
    return res


def map2alm_ms(geom, m_, lmax: int, ms) -> list:
    """Separable analysis (Section 2.2) for the selected m: list of a_{l m}, l = m..lmax."""
    d = delta_anal(geom, m_, ms)
    return legendre_anal(geom, d, lmax, ms)


def map2alm_rings(geom, m_, lmax: int, mmax: int) -> np.ndarray:
    """Separable analysis for every m, as a full m-major coefficient vector."""
    ms = np.arange(mmax + 1)
    parts = map2alm_ms(geom, m_, lmax, ms)
    return np.concatenate(parts)


# ---------------------------------------------------------------- spin-weighted (spin 2)
#
# Polarisation maps (Q, U) and coefficients (E, B) as defined at the top of spin_oracle.c:
# Q + iU = sum 2a_lm 2Y_lm with 2a_lm = -(E_lm + i B_lm), the analysis with conj(Y) and the ring
# weights.  Arrays: E, B complex m-major triangles (the first l = 0, 1 entries are ignored on input
# and zero on output); Q, U real [npix] in ring order.


def spin_lambda(theta: float, lmax: int, m: int, s: int) -> np.ndarray:
    """slambda_{l m}(theta) for l = m..lmax (zero for l < max(m, |s|))."""
    out = np.zeros(lmax - m + 1, dtype=np.float64)
    _load().oracle_spin_lambda(float(theta), int(lmax), int(m), int(s), _p(out))
    return out


def spin_delta_synth(geom, E, B, lmax: int, mmax: int, rings=None):
    """Delta^Q_m(r), Delta^U_m(r) of the spin-2 synthesis, each [len(rings)][mmax+1] complex."""
    nphi, theta, phi0, w = geom
    theta = _f64(theta)
    rings = _i32(np.arange(len(theta)) if rings is None else rings)
    E, B = _c128(E), _c128(B)
    assert E.size == nalm(lmax, mmax) and B.size == E.size
    dq = np.zeros((len(rings), mmax + 1), dtype=np.complex128)
    du = np.zeros_like(dq)
    _load().oracle_spin_delta_synth(len(theta), _p(theta), lmax, mmax, _p(E), _p(B), len(rings), _p(rings),
                                    _p(dq), _p(du))
    return dq, du


def spin_alm2map_rings(geom, E, B, lmax: int, mmax: int, rings=None):
    """Separable spin-2 synthesis of the selected rings: (Q, U) pixels, concatenated by ring."""
    rings = np.arange(len(geom[0])) if rings is None else np.asarray(rings)
    dq, du = spin_delta_synth(geom, E, B, lmax, mmax, rings)
    return ring_synth(geom, dq, mmax, rings), ring_synth(geom, du, mmax, rings)


def spin_map2alm_ms(geom, q, u, lmax: int, ms):
    """Separable spin-2 analysis for the selected m: lists of E_{l m} and B_{l m}, l = m..lmax."""
    nphi, theta, phi0, w = geom
    theta = _f64(theta)
    ms = _i32(ms)
    dq = delta_anal(geom, q, ms)
    du = delta_anal(geom, u, ms)
    sizes = [lmax - int(m) + 1 for m in ms]
    E = np.zeros(sum(sizes), dtype=np.complex128)
    B = np.zeros_like(E)
    _load().oracle_spin_legendre_anal(len(theta), _p(theta), lmax, len(ms), _p(ms), _p(_c128(dq)), _p(_c128(du)),
                                      _p(E), _p(B))
    outE, outB, o = [], [], 0
    for sz in sizes:
        outE.append(E[o:o + sz].copy())
        outB.append(B[o:o + sz].copy())
        o += sz
    return outE, outB


def spin_map2alm_rings(geom, q, u, lmax: int, mmax: int):
    """Separable spin-2 analysis for every m, as full m-major E and B vectors."""
    E, B = spin_map2alm_ms(geom, q, u, lmax, np.arange(mmax + 1))
    return np.concatenate(E), np.concatenate(B)


def spin_alm2map_exact(geom, E, B, lmax: int, mmax: int):
    """Pixel-by-pixel spin-2 synthesis from the definition: (Q, U)."""
    nphi, theta, phi0, w = geom
    nphi, theta, phi0 = _i64(nphi), _f64(theta), _f64(phi0)
    E, B = _c128(E), _c128(B)
    assert E.size == nalm(lmax, mmax) and B.size == E.size
    q = np.zeros(int(nphi.sum()), dtype=np.float64)
    u = np.zeros_like(q)
    _load().oracle_spin_alm2map_exact(len(nphi), _p(nphi), _p(theta), _p(phi0), lmax, mmax, _p(E), _p(B), _p(q), _p(u))
    return q, u


def spin_map2alm_exact(geom, q, u, lmax: int, mmax: int):
    """Pixel-by-pixel spin-2 analysis from the definition: (E, B)."""
    nphi, theta, phi0, w = geom
    nphi, theta, phi0, w = _i64(nphi), _f64(theta), _f64(phi0), _f64(w)
    q, u = _f64(q), _f64(u)
    assert q.size == nphi.sum() and u.size == q.size
    E = np.zeros(nalm(lmax, mmax), dtype=np.complex128)
    B = np.zeros_like(E)
    _load().oracle_spin_map2alm_exact(len(nphi), _p(nphi), _p(theta), _p(phi0), _p(w), lmax, mmax, _p(q), _p(u),
                                      _p(E), _p(B))
    return E, B
