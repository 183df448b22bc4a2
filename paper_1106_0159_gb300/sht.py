"""Python binding of the C ABI in ``include/sht.h`` (argument marshalling only).

Every transform step runs in the CUDA library ``_lib/libsht.so``; this module
only checks tensor shapes, passes device pointers and the current CUDA
stream, and turns status codes into exceptions.  There is no CPU path: if
the library cannot be loaded the calls raise.

PyTorch supplies device memory and streams.  Coefficients are complex128
tensors of shape [nmaps, nalm] in m-major triangular order, maps float64
tensors of shape [nmaps, npix], Delta intermediates complex128
[nmaps, nrings, mmax + 1].
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libsht.so")
_lock = threading.Lock()
_lib = None

SHT_OK, SHT_EINVAL, SHT_ENOMEM, SHT_ECUDA, SHT_EUNSUPPORTED, SHT_ETIMEOUT = range(6)
GRID_CUSTOM, GRID_HEALPIX, GRID_GAUSS_LEGENDRE = 0, 1, 2

# every entry point the header declares (the test suite checks the library exports them)
EXPORTS = (
    "sht_plan_create", "sht_plan_destroy", "sht_alm2map", "sht_map2alm",
    "sht_legendre_synth", "sht_ring_synth", "sht_ring_anal", "sht_legendre_anal",
    "sht_nalm", "sht_alm_index", "sht_plan_npix", "sht_plan_nrings", "sht_plan_npairs",
    "sht_workspace_bytes", "sht_geom_healpix", "sht_geom_gauss_legendre",
    "sht_status_string", "sht_plan_last_error", "sht_plan_set_stage_timing", "sht_plan_stage_times",
    "sht_fp64_fma_tflops", "sht_alm2map_noalloc", "sht_noalloc_scratch_bytes",
    "sht_plan_set_mode", "sht_plan_mode", "sht_plan_device_status", "sht_plan_reserve",
    "sht_plan_set_tuning", "sht_plan_tuning", "sht_plan_selftest_timeout", "sht_alm2map_ws", "sht_map2alm_ws",
    "sht_plan_live_steps", "sht_alm2map_spin", "sht_map2alm_spin", "sht_spin_workspace_bytes",
    "sht_plan_set_mlist", "sht_debug_fail_allocations_after",
    "sht_batch_create", "sht_batch_set_tuning", "sht_batch_tuning", "sht_batch_run", "sht_batch_tiles",
    "sht_batch_last_error", "sht_batch_destroy",
)
MODE_FP64, MODE_SPLIT_BF16 = 0, 1
# launch tuning knobs (sht_tune) and the values each takes
(TUNE_SYNTH_MAPS, TUNE_ANAL_MAPS, TUNE_ANAL_SLOTS, TUNE_DF_MAPS, TUNE_TC_MAPS, TUNE_PREC_ANAL, TUNE_PREC_RING,
 TUNE_RING_SMEM) = range(8)
TUNE_VALUES = {TUNE_SYNTH_MAPS: (1, 2, 4), TUNE_ANAL_MAPS: (1, 2), TUNE_ANAL_SLOTS: (1, 4),
               TUNE_DF_MAPS: (4, 8, 16), TUNE_TC_MAPS: (8, 16), TUNE_PREC_ANAL: (0, 1), TUNE_PREC_RING: (0, 1),
               TUNE_RING_SMEM: (0, 1, 2)}
STAGES = ("legendre_synth", "ring_synth", "ring_anal", "legendre_anal", "block_reduce", "tc_synth_kernel",
          "tc_anal_kernel")


class ShtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load (building first if absent or stale) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import _build
        _build.build()
        lib = ctypes.CDLL(_LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        S = ctypes.c_size_t
        sig = {
            "sht_plan_create": (I, [ctypes.POINTER(P), I, I, P, P, P, P, I, I]),
            "sht_plan_destroy": (None, [P]),
            "sht_alm2map": (I, [P, P, P, I, P]),
            "sht_map2alm": (I, [P, P, P, I, P]),
            "sht_legendre_synth": (I, [P, P, P, I, P]),
            "sht_ring_synth": (I, [P, P, P, I, P]),
            "sht_ring_anal": (I, [P, P, P, I, P]),
            "sht_legendre_anal": (I, [P, P, P, I, P]),
            "sht_nalm": (I64, [I, I]),
            "sht_alm_index": (I64, [I, I, I]),
            "sht_plan_npix": (I64, [P]),
            "sht_plan_nrings": (I, [P]),
            "sht_plan_npairs": (I, [P]),
            "sht_workspace_bytes": (S, [P, I]),
            "sht_geom_healpix": (I, [I, P, P, P, P]),
            "sht_geom_gauss_legendre": (I, [I, I64, P, P, P, P]),
            "sht_status_string": (ctypes.c_char_p, [I]),
            "sht_plan_last_error": (ctypes.c_char_p, [P]),
            "sht_plan_set_stage_timing": (I, [P, I]),
            "sht_plan_stage_times": (I, [P, P, P, I]),
            "sht_fp64_fma_tflops": (I, [P]),
            "sht_alm2map_noalloc": (I, [P, P, P, I, P]),
            "sht_noalloc_scratch_bytes": (S, []),
            "sht_plan_set_mode": (I, [P, I]),
            "sht_plan_mode": (I, [P]),
            "sht_plan_live_steps": (I, [P, P, P]),
            "sht_alm2map_spin": (I, [P, I, P, P, I, P]),
            "sht_map2alm_spin": (I, [P, I, P, P, I, P]),
            "sht_spin_workspace_bytes": (S, [P, I]),
            "sht_plan_set_mlist": (I, [P, P, I]),
            "sht_debug_fail_allocations_after": (ctypes.c_long, [ctypes.c_long]),
            "sht_batch_create": (I, [ctypes.POINTER(P), I, I, P, P, P, P]),
            "sht_batch_set_tuning": (I, [P, I, I]),
            "sht_batch_tuning": (I, [P, I]),
            "sht_batch_run": (I, [P, P]),
            "sht_batch_tiles": (I64, [P, I]),
            "sht_batch_last_error": (ctypes.c_char_p, [P]),
            "sht_batch_destroy": (None, [P]),
            "sht_plan_device_status": (I, [P, P, I]),
            "sht_plan_reserve": (I, [P, I]),
            "sht_plan_set_tuning": (I, [P, I, I]),
            "sht_plan_tuning": (I, [P, I]),
            "sht_plan_selftest_timeout": (I, [P, P]),
            "sht_alm2map_ws": (I, [P, P, P, I, P, P, S]),
            "sht_map2alm_ws": (I, [P, P, P, I, P, P, S]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status: int, plan_ptr=None, what: str = ""):
    if status == SHT_OK:
        return
    lib = load()
    msg = lib.sht_status_string(status).decode()
    if plan_ptr:
        extra = lib.sht_plan_last_error(plan_ptr).decode()
        if extra:
            msg += ": " + extra
    if what:
        msg = what + ": " + msg
    if status == SHT_EINVAL:
        raise ValueError(msg)
    raise ShtError(status, msg)


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def nalm(lmax: int, mmax: int) -> int:
    return int(load().sht_nalm(int(lmax), int(mmax)))


def alm_index(lmax: int, l: int, m: int) -> int:
    return int(load().sht_alm_index(int(lmax), int(l), int(m)))


def healpix_geometry(nside: int):
    """(nphi, theta, phi0, w) of the HEALPix grid, from the library's host helper."""
    nr = 4 * int(nside) - 1
    if nr < 3:
        raise ValueError("nside must be >= 1")
    nphi = np.zeros(nr, np.int64)
    th, p0, w = (np.zeros(nr) for _ in range(3))
    _check(load().sht_geom_healpix(int(nside), _np_ptr(nphi), _np_ptr(th), _np_ptr(p0), _np_ptr(w)), what="healpix")
    return nphi, th, p0, w


def gauss_legendre_geometry(nrings: int, nphi: int):
    """(nphi, theta, phi0, w) of a Gauss-Legendre grid, from the library's host helper."""
    if int(nrings) < 1:
        raise ValueError("nrings must be >= 1")
    n = np.zeros(int(nrings), np.int64)
    th, p0, w = (np.zeros(int(nrings)) for _ in range(3))
    _check(load().sht_geom_gauss_legendre(int(nrings), int(nphi), _np_ptr(n), _np_ptr(th), _np_ptr(p0), _np_ptr(w)),
           what="gauss_legendre")
    return n, th, p0, w


def fp64_fma_tflops() -> float:
    """Measured FP64 FMA throughput of the current GPU (TFLOP/s)."""
    v = ctypes.c_double()
    _check(load().sht_fp64_fma_tflops(ctypes.byref(v)), what="sht_fp64_fma_tflops")
    return float(v.value)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A transform plan: ring geometry and band limits, with device tables.

    ``geom`` is (nphi, theta, phi0, w) per ring (host arrays, copied).
    """

    def __init__(self, geom, lmax: int, mmax: int | None = None, grid: int = GRID_CUSTOM):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the spherical harmonic transforms need a CUDA device")
        torch.cuda.init()
        lib = load()
        mmax = int(lmax) if mmax is None else int(mmax)
        nphi, theta, phi0, w = geom
        self._nphi = np.ascontiguousarray(nphi, dtype=np.int64)
        self._theta = np.ascontiguousarray(theta, dtype=np.float64)
        self._phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        self._w = np.ascontiguousarray(w, dtype=np.float64)
        n = len(self._nphi)
        if not (len(self._theta) == len(self._phi0) == len(self._w) == n):
            raise ValueError("geometry arrays differ in length")
        h = ctypes.c_void_p()
        st = lib.sht_plan_create(ctypes.byref(h), int(grid), n, _np_ptr(self._nphi), _np_ptr(self._theta),
                                 _np_ptr(self._phi0), _np_ptr(self._w), int(lmax), mmax)
        _check(st, what="sht_plan_create")
        self._h = h
        self.lmax, self.mmax = int(lmax), mmax
        self.nrings = n
        self.npix = int(lib.sht_plan_npix(h))
        self.nalm = nalm(lmax, mmax)
        self.npairs = int(lib.sht_plan_npairs(h))

    def close(self):
        if getattr(self, "_h", None):
            load().sht_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode: int):
        """MODE_FP64 (default) or MODE_SPLIT_BF16 (the precision form: tensor-core sums over l and rings)."""
        _check(load().sht_plan_set_mode(self._h, int(mode)), self._h, "sht_plan_set_mode")

    @property
    def mode(self) -> int:
        return int(load().sht_plan_mode(self._h))

    def device_status(self, clear: bool = True) -> int:
        """The plan's device status word (bit 0: a bounded device wait gave up); waits for the device."""
        v = ctypes.c_int()
        st = load().sht_plan_device_status(self._h, ctypes.byref(v), 1 if clear else 0)
        if st != SHT_ETIMEOUT:
            _check(st, self._h)
        return int(v.value)

    def set_mlist(self, ms=None):
        """Restrict the FP64 Legendre steps to the listed m (None or empty: every m)."""
        arr = np.ascontiguousarray([] if ms is None else ms, dtype=np.int32)
        ptr = _np_ptr(arr) if arr.size else None
        _check(load().sht_plan_set_mlist(self._h, ptr, int(arr.size)), self._h, "sht_plan_set_mlist")

    def live_steps(self):
        """(live, total) recurrence steps of one pass: total = nalm * slots; live from the first
        32-l chunk per (m, 128-slot block) with a value above the dropping threshold (needs the
        precision-form tables: call set_mode(MODE_SPLIT_BF16) once first)."""
        lv, tot = ctypes.c_int64(), ctypes.c_int64()
        _check(load().sht_plan_live_steps(self._h, ctypes.byref(lv), ctypes.byref(tot)), self._h)
        return int(lv.value), int(tot.value)

    def selftest_timeout(self, stream=None):
        """Run the failure path of the device waits once (sets bit 0 of the status word)."""
        _check(load().sht_plan_selftest_timeout(self._h, _stream_ptr(stream)), self._h)

    def set_stage_timing(self, enable: bool):
        _check(load().sht_plan_set_stage_timing(self._h, 1 if enable else 0), self._h)

    def stage_times(self, reset: bool = False):
        """{stage: (ms, launches)} accumulated since the last reset (waits for the recorded events)."""
        ms = np.zeros(len(STAGES), np.float64)
        nl = np.zeros(len(STAGES), np.int64)
        _check(load().sht_plan_stage_times(self._h, _np_ptr(ms), _np_ptr(nl), 1 if reset else 0), self._h)
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(STAGES)}

    def workspace_bytes(self, nmaps: int) -> int:
        return int(load().sht_workspace_bytes(self._h, int(nmaps)))

    def set_tuning(self, knob: int, value: int):
        """Set a launch-tuning knob (TUNE_*); see TUNE_VALUES for what each takes."""
        _check(load().sht_plan_set_tuning(self._h, int(knob), int(value)), self._h, "sht_plan_set_tuning")

    def tuning(self, knob: int) -> int:
        return int(load().sht_plan_tuning(self._h, int(knob)))

    def reserve(self, nmaps: int):
        """Grow the plan's device scratch now so calls with <= nmaps maps allocate nothing."""
        _check(load().sht_plan_reserve(self._h, int(nmaps)), self._h, "sht_plan_reserve")

    # -- tensor checks ------------------------------------------------------
    def _dev(self, t, dtype, tail, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if t.dim() == len(tail):
            t = t.unsqueeze(0)
        if tuple(t.shape[1:]) != tuple(tail):
            raise ValueError("%s has shape %s, expected [nmaps, %s]" % (name, tuple(t.shape), tail))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return t

    def _out(self, out, shape, dtype, like):
        import torch
        if out is None:
            return torch.empty(shape, dtype=dtype, device=like.device)
        o = self._dev(out, dtype, shape[1:], "out")
        if o.shape[0] != shape[0]:
            raise ValueError("out has %d maps, expected %d" % (o.shape[0], shape[0]))
        return o

    def _run(self, fn, src, dst, nmaps, stream):
        st = fn(self._h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), int(nmaps),
                _stream_ptr(stream))
        _check(st, self._h, fn.__name__)

    # -- transforms ---------------------------------------------------------
    def alm2map(self, alm, out=None, stream=None):
        """Synthesis (Algorithm 2): [nmaps, nalm] complex128 -> [nmaps, npix] float64."""
        import torch
        a = self._dev(alm, torch.complex128, (self.nalm,), "alm")
        o = self._out(out, (a.shape[0], self.npix), torch.float64, a)
        self._run(load().sht_alm2map, a, o, a.shape[0], stream)
        return o

    def alm2map_noalloc(self, alm, out=None, stream=None):
        """Synthesis through sht_alm2map_noalloc: the library call itself allocates no device
        memory (its scratch is a static device array); only `out`, if not given, is allocated
        here by PyTorch before the call."""
        import torch
        a = self._dev(alm, torch.complex128, (self.nalm,), "alm")
        o = self._out(out, (a.shape[0], self.npix), torch.float64, a)
        self._run(load().sht_alm2map_noalloc, a, o, a.shape[0], stream)
        return o

    def map2alm(self, m, out=None, stream=None):
        """Analysis (Algorithm 1): [nmaps, npix] float64 -> [nmaps, nalm] complex128."""
        import torch
        s = self._dev(m, torch.float64, (self.npix,), "map")
        o = self._out(out, (s.shape[0], self.nalm), torch.complex128, s)
        self._run(load().sht_map2alm, s, o, s.shape[0], stream)
        return o

    def alm2map_spin(self, alm, out=None, stream=None, spin: int = 2):
        """Spin-2 synthesis: [nmaps, 2, nalm] complex128 (E, B) -> [nmaps, 2, npix] float64 (Q, U)."""
        import torch
        a = self._dev(alm, torch.complex128, (2, self.nalm), "alm")
        o = self._out(out, (a.shape[0], 2, self.npix), torch.float64, a)
        st = load().sht_alm2map_spin(self._h, int(spin), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                     int(a.shape[0]), _stream_ptr(stream))
        _check(st, self._h, "sht_alm2map_spin")
        return o

    def map2alm_spin(self, m, out=None, stream=None, spin: int = 2):
        """Spin-2 analysis: [nmaps, 2, npix] float64 (Q, U) -> [nmaps, 2, nalm] complex128 (E, B)."""
        import torch
        s = self._dev(m, torch.float64, (2, self.npix), "map")
        o = self._out(out, (s.shape[0], 2, self.nalm), torch.complex128, s)
        st = load().sht_map2alm_spin(self._h, int(spin), ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                     int(s.shape[0]), _stream_ptr(stream))
        _check(st, self._h, "sht_map2alm_spin")
        return o

    def scratch(self, nmaps: int):
        """A device scratch buffer for the *_ws calls with up to nmaps maps (uint8 tensor)."""
        import torch
        return torch.empty((self.workspace_bytes(nmaps),), dtype=torch.uint8, device="cuda")

    def _run_ws(self, fn, src, dst, nmaps, stream, scratch):
        if not (hasattr(scratch, "is_cuda") and scratch.is_cuda):
            raise TypeError("scratch must be a CUDA tensor")
        st = fn(self._h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), int(nmaps),
                _stream_ptr(stream), ctypes.c_void_p(scratch.data_ptr()),
                ctypes.c_size_t(scratch.numel() * scratch.element_size()))
        _check(st, self._h, fn.__name__)

    def alm2map_ws(self, alm, scratch, out=None, stream=None):
        """alm2map on caller scratch (from scratch()): one plan can serve several streams."""
        import torch
        a = self._dev(alm, torch.complex128, (self.nalm,), "alm")
        o = self._out(out, (a.shape[0], self.npix), torch.float64, a)
        self._run_ws(load().sht_alm2map_ws, a, o, a.shape[0], stream, scratch)
        return o

    def map2alm_ws(self, m, scratch, out=None, stream=None):
        """map2alm on caller scratch (from scratch())."""
        import torch
        s = self._dev(m, torch.float64, (self.npix,), "map")
        o = self._out(out, (s.shape[0], self.nalm), torch.complex128, s)
        self._run_ws(load().sht_map2alm_ws, s, o, s.shape[0], stream, scratch)
        return o

    def legendre_synth(self, alm, out=None, stream=None):
        import torch
        a = self._dev(alm, torch.complex128, (self.nalm,), "alm")
        o = self._out(out, (a.shape[0], self.nrings, self.mmax + 1), torch.complex128, a)
        self._run(load().sht_legendre_synth, a, o, a.shape[0], stream)
        return o

    def ring_synth(self, delta, out=None, stream=None):
        import torch
        d = self._dev(delta, torch.complex128, (self.nrings, self.mmax + 1), "delta")
        o = self._out(out, (d.shape[0], self.npix), torch.float64, d)
        self._run(load().sht_ring_synth, d, o, d.shape[0], stream)
        return o

    def ring_anal(self, m, out=None, stream=None):
        import torch
        s = self._dev(m, torch.float64, (self.npix,), "map")
        o = self._out(out, (s.shape[0], self.nrings, self.mmax + 1), torch.complex128, s)
        self._run(load().sht_ring_anal, s, o, s.shape[0], stream)
        return o

    def legendre_anal(self, delta, out=None, stream=None):
        import torch
        d = self._dev(delta, torch.complex128, (self.nrings, self.mmax + 1), "delta")
        o = self._out(out, (d.shape[0], self.nalm), torch.complex128, d)
        self._run(load().sht_legendre_anal, d, o, d.shape[0], stream)
        return o


# batched form: knobs of sht_batch_set_tuning and the values each takes
BATCH_SYNTH_MAPS, BATCH_LEG_CTAS, BATCH_RING_CTAS, BATCH_ANAL_MAPS, BATCH_ANAL_SLOTS = range(5)
BATCH_TUNE_VALUES = {BATCH_SYNTH_MAPS: (1, 2, 4), BATCH_LEG_CTAS: (2, 4, 8, 16), BATCH_RING_CTAS: (1, 2, 3, 4),
                     BATCH_ANAL_MAPS: (1, 2), BATCH_ANAL_SLOTS: (1, 4)}
BATCH_ALM2MAP, BATCH_MAP2ALM = 0, 1


class Batch:
    """Many transforms of one direction as one persistent launch per stage (sht_batch_*).

    jobs: list of (plan, src, dst) with the tensors of plan.alm2map / plan.map2alm (device,
    contiguous, kept by the batch: write new inputs into src in place between runs)."""

    def __init__(self, direction: int, jobs):
        import torch
        self.direction = int(direction)
        self.jobs = list(jobs)
        chk = []
        for plan, src, dst in self.jobs:
            if self.direction == BATCH_ALM2MAP:
                a = plan._dev(src, torch.complex128, (plan.nalm,), "alm")
                o = plan._dev(dst, torch.float64, (plan.npix,), "map")
            else:
                a = plan._dev(src, torch.float64, (plan.npix,), "map")
                o = plan._dev(dst, torch.complex128, (plan.nalm,), "alm")
            if a.shape[0] != o.shape[0]:
                raise ValueError("src and dst map counts differ")
            chk.append((plan, a, o))
        self.jobs = chk
        n = len(chk)
        P = ctypes.c_void_p
        plans = (P * n)(*[P(p._h.value if hasattr(p._h, "value") else p._h) for p, _, _ in chk])
        ins = (P * n)(*[P(a.data_ptr()) for _, a, _ in chk])
        outs = (P * n)(*[P(o.data_ptr()) for _, _, o in chk])
        nm = (ctypes.c_int * n)(*[int(a.shape[0]) for _, a, _ in chk])
        self._h = P()
        _check(load().sht_batch_create(ctypes.byref(self._h), self.direction, n, plans, ins, outs, nm), None,
               "sht_batch_create")

    def _err(self, st, what):
        if st != SHT_OK:
            extra = load().sht_batch_last_error(self._h).decode()
            msg = what + ": " + load().sht_status_string(st).decode() + (": " + extra if extra else "")
            if st == SHT_EINVAL:
                raise ValueError(msg)
            raise ShtError(st, msg)

    def set_tuning(self, knob: int, value: int):
        self._err(load().sht_batch_set_tuning(self._h, int(knob), int(value)), "sht_batch_set_tuning")

    def tuning(self, knob: int) -> int:
        return int(load().sht_batch_tuning(self._h, int(knob)))

    def run(self, stream=None):
        self._err(load().sht_batch_run(self._h, _stream_ptr(stream)), "sht_batch_run")

    def tiles(self, stage: int) -> int:
        return int(load().sht_batch_tiles(self._h, int(stage)))

    def close(self):
        if self._h:
            load().sht_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
