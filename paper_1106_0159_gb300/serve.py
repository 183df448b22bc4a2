"""Continuous-batching server for alm2map / map2alm requests.

Requests of different band limits and map counts arrive over time.  The
server keeps plans and data on the device and groups pending requests that
share a plan and a direction into batches of up to `max_batch_maps` maps
(one transform call runs all of them; the maps are independent, so a
request's result does not depend on its batch mates).  A batch is admitted
when a stream is free and its device memory (inputs, outputs and the plan's
scratch) fits the memory budget; batches on different streams overlap on
the GPU.  Each request records its arrival and completion times, from which
the server reports p50/p99 latency and throughput.

Memory model: the plans (tables and their scratch, grown once to the largest
batch at warm-up) stay resident and are counted once; each batch in flight
adds its inputs and outputs.  A batch waits while the resident bytes plus the
bytes in flight plus its own would exceed the budget, unless nothing is in
flight (an idle server always admits, so every request makes progress).

A pending request can be cancelled, and one whose deadline passes before it
is admitted is dropped with status "timeout"; a request already on the GPU
runs to the end (no kernel is interrupted) and a cancellation then only
discards its result.  With ``batching=False`` and one stream the server is the
plain one-at-a-time path: each request is one call, in arrival order.

The transforms themselves run in the CUDA library (``sht.Plan``, one plan
per grid and band limit shared by the stream slots, each slot with its own
scratch); this module only schedules.  The backend is injectable so the scheduling logic
can be exercised without a GPU (``tests/test_serve.py``).
"""
from __future__ import annotations

import collections
import dataclasses
import itertools
import statistics
import time
from typing import Any, Callable, Dict, List, Optional, Tuple

ALM2MAP, MAP2ALM = "alm2map", "map2alm"


@dataclasses.dataclass(eq=False)
class Request:
    direction: str            # ALM2MAP or MAP2ALM
    lmax: int
    nside: int                # HEALPix grid of the request
    data: Any                 # [nmaps, nalm] complex128 (alm2map) or [nmaps, npix] float64 (map2alm)
    nmaps: int
    arrival: float = 0.0      # seconds, server clock
    deadline: Optional[float] = None  # seconds after arrival; dropped if not admitted by then
    rid: int = -1
    status: str = "new"       # new, pending, running, done, cancelled, timeout
    start: Optional[float] = None
    done: Optional[float] = None
    result: Any = None

    @property
    def key(self) -> Tuple[int, int]:
        return (self.nside, self.lmax)

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


@dataclasses.dataclass(eq=False)
class Batch:
    key: Tuple[int, int]
    direction: str
    requests: List[Request]
    stream_slot: int
    nbytes: int
    handle: Any = None

    @property
    def nmaps(self) -> int:
        return sum(r.nmaps for r in self.requests)


class Server:
    """Scheduler.  Drive it with submit() and poll() (or run_trace() for a timed arrival trace)."""

    def __init__(self, backend, max_batch_maps: int = 32, nstreams: int = 2, memory_budget: Optional[int] = None,
                 batching: bool = True, clock: Callable[[], float] = time.perf_counter, keep_results: bool = True):
        self.backend = backend
        self.keep_results = bool(keep_results)   # False: a finished request keeps its times, not its output
        self.max_batch_maps = int(max_batch_maps)
        self.nstreams = int(nstreams)
        self.batching = bool(batching)
        self.budget = memory_budget if memory_budget is not None else backend.memory_budget()
        self.clock = clock
        self.pending: "collections.deque[Request]" = collections.deque()
        self.running: Dict[int, Batch] = {}
        self.completed: List[Request] = []
        self.dropped: List[Request] = []
        self.bytes_in_flight = 0
        self._ids = itertools.count()
        self.nbatches = 0

    # -- requests -----------------------------------------------------------
    def submit(self, req: Request, arrival: Optional[float] = None) -> Request:
        if req.direction not in (ALM2MAP, MAP2ALM):
            raise ValueError("unknown direction %r" % (req.direction,))
        if req.nmaps < 1:
            raise ValueError("a request carries at least one map")
        req.rid = next(self._ids)
        req.arrival = self.clock() if arrival is None else arrival
        req.status = "pending"
        self.pending.append(req)
        return req

    def cancel(self, req: Request) -> bool:
        """Cancel a request.  True if it was still pending (it will not run); a running request
        finishes on the GPU and its result is discarded; a finished one is left as it is."""
        if req.status == "pending":
            self.pending.remove(req)
            req.status = "cancelled"
            self.dropped.append(req)
            return True
        if req.status == "running":
            req.status = "cancelled"
        return False

    def _expire(self, now: float) -> None:
        for r in list(self.pending):
            if r.deadline is not None and now - r.arrival > r.deadline:
                self.pending.remove(r)
                r.status = "timeout"
                self.dropped.append(r)

    # -- scheduling ---------------------------------------------------------
    def _form_batch(self) -> Optional[List[Request]]:
        """Oldest pending request plus later ones with the same plan and direction, FIFO order."""
        if not self.pending:
            return None
        head = self.pending[0]
        if not self.batching:
            return [head]
        # The oldest request always goes (alone if it exceeds the batch size), so none starves.
        chosen, total = [head], head.nmaps
        for r in itertools.islice(self.pending, 1, None):
            if total >= self.max_batch_maps:
                break
            if r.key == head.key and r.direction == head.direction and total + r.nmaps <= self.max_batch_maps:
                chosen.append(r)
                total += r.nmaps
        return chosen

    def _free_slot(self) -> Optional[int]:
        for s in range(self.nstreams):
            if s not in self.running:
                return s
        return None

    def poll(self) -> int:
        """Retire finished batches, then admit new ones while a stream and memory are free.
        Returns the number of requests completed by this call."""
        finished = 0
        for slot, b in list(self.running.items()):
            if self.backend.done(b.handle):
                outs = self.backend.results(b.handle)
                t = self.clock()
                for r, o in zip(b.requests, outs):
                    r.done = t
                    if r.status == "cancelled":
                        self.dropped.append(r)
                        continue
                    r.result = o if self.keep_results else None
                    r.status = "done"
                    self.completed.append(r)
                    finished += 1
                self.bytes_in_flight -= b.nbytes
                del self.running[slot]
        self._expire(self.clock())
        while True:
            slot = self._free_slot()
            if slot is None:
                break
            reqs = self._form_batch()
            if reqs is None:
                break
            head = reqs[0]
            nmaps = sum(r.nmaps for r in reqs)
            nbytes = self.backend.batch_bytes(head.key, head.direction, nmaps)
            if self.running and self.backend.resident_bytes() + self.bytes_in_flight + nbytes > self.budget:
                break  # wait for memory; an idle server admits anything (it must make progress)
            for r in reqs:
                self.pending.remove(r)
            t = self.clock()
            for r in reqs:
                r.start = t
                r.status = "running"
            b = Batch(head.key, head.direction, reqs, slot, nbytes)
            b.handle = self.backend.launch(head.key, head.direction, [r.data for r in reqs],
                                           [r.nmaps for r in reqs], slot)
            self.bytes_in_flight += nbytes
            self.running[slot] = b
            self.nbatches += 1
        return finished

    def idle(self) -> bool:
        return not self.pending and not self.running

    def drain(self, timeout: float = 600.0) -> None:
        t0 = self.clock()
        while not self.idle():
            self.poll()
            if self.clock() - t0 > timeout:
                raise TimeoutError("requests still pending after %.0f s" % timeout)

    def run_trace(self, trace: List[Tuple[float, Request]], timeout: float = 600.0) -> None:
        """Replay (offset seconds, request) pairs: each request is submitted when the server clock
        passes its offset from the start; the loop polls continuously in between."""
        trace = sorted(trace, key=lambda x: x[0])
        t0 = self.clock()
        i = 0
        while i < len(trace) or not self.idle():
            now = self.clock() - t0
            while i < len(trace) and trace[i][0] <= now:
                self.submit(trace[i][1], arrival=t0 + trace[i][0])
                i += 1
            self.poll()
            if now > timeout:
                raise TimeoutError("trace did not finish in %.0f s" % timeout)

    # -- statistics ---------------------------------------------------------
    def stats(self) -> Dict[str, float]:
        lat = sorted(r.latency for r in self.completed if r.latency is not None)
        if not lat:
            return {"requests": 0}
        t_first = min(r.arrival for r in self.completed)
        t_last = max(r.done for r in self.completed)
        maps = sum(r.nmaps for r in self.completed)
        return {"requests": len(lat), "maps": maps, "batches": self.nbatches, "dropped": len(self.dropped),
                "wall_s": t_last - t_first, "maps_per_s": maps / max(t_last - t_first, 1e-12),
                "p50_ms": 1e3 * statistics.median(lat), "p99_ms": 1e3 * _percentile(lat, 0.99),
                "max_ms": 1e3 * lat[-1]}


def _percentile(sorted_vals, q):
    if not sorted_vals:
        return float("nan")
    k = min(len(sorted_vals) - 1, max(0, int(round(q * (len(sorted_vals) - 1)))))
    return sorted_vals[k]


# ---------------------------------------------------------------- GPU backend

class TorchBackend:
    """Runs batches with the CUDA library: one plan per (grid, band limit), kept on the device and
    shared by the stream slots.  Each stream slot owns one scratch buffer, sized for the largest
    plan and used by whichever plan its batch needs (sht_alm2map_ws / sht_map2alm_ws): a slot runs
    one batch at a time, so the scratch grows with the slots, not with the number of plans.  Inputs
    are concatenated on the device, one transform call per batch, results split back per request
    (device tensors)."""

    def __init__(self, mode: int = 1, device=None, nstreams: int = 2, budget_fraction: float = 0.8):
        import torch

        from . import sht
        self.torch = torch
        self.sht = sht
        self.mode = mode
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(nstreams)]
        self.plans: Dict[Tuple[int, int], Any] = {}
        self.scratch: Dict[int, Any] = {}        # stream slot -> scratch buffer
        self.resident: Dict[Any, int] = {}
        self.budget_fraction = budget_fraction

    def memory_budget(self) -> int:
        _, total = self.torch.cuda.mem_get_info(self.device)
        return int(total * self.budget_fraction)

    def plan(self, key, slot=0):
        """The plan of a (nside, lmax) key, shared by every stream slot."""
        p = self.plans.get(key)
        if p is None:
            nside, lmax = key
            p = self.sht.Plan(self.sht.healpix_geometry(nside), lmax, lmax, grid=self.sht.GRID_HEALPIX)
            p.set_mode(self.mode)
            self.plans[key] = p
        return p

    def warm(self, keys, max_maps: int):
        """Create every plan and the scratch of every (plan, stream slot) for `max_maps` maps, so
        that nothing is allocated while serving, and run small transforms (1 and 17 maps, both
        directions) on the smallest plan so that every kernel is loaded before the first request.
        Returns the seconds it took (plan creation is not serving)."""
        torch = self.torch
        t0 = time.perf_counter()
        need = 0
        for key in keys:
            p = self.plan(key)
            self.resident[key] = 0
            need = max(need, p.workspace_bytes(max_maps))
        for slot in range(len(self.streams)):
            self._grow(slot, need)
        small = min(keys, key=lambda k: k[1])
        p = self.plan(small)
        for n in (1, 17):
            if n > max_maps:
                continue
            a = torch.zeros((n, p.nalm), dtype=torch.complex128, device=self.device)
            p.map2alm_ws(p.alm2map_ws(a, self.scratch[0]), self.scratch[0])
        torch.cuda.synchronize(self.device)
        return time.perf_counter() - t0

    def close(self):
        """Release every plan (tables) and scratch buffer."""
        self.torch.cuda.synchronize(self.device)
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        self.scratch.clear()
        self.resident.clear()
        self.torch.cuda.empty_cache()

    def _grow(self, slot, nbytes):
        cur = self.scratch.get(slot)
        if cur is None or cur.numel() < nbytes:
            self.scratch[slot] = None
            self.torch.cuda.synchronize(self.device)   # the old buffer may still be read by the slot's stream
            self.scratch[slot] = self.torch.empty((int(nbytes),), dtype=self.torch.uint8, device=self.device)
            self.resident[("scratch", slot)] = int(nbytes)
        return self.scratch[slot]

    def resident_bytes(self) -> int:
        return sum(self.resident.values())

    def batch_bytes(self, key, direction, nmaps) -> int:
        p = self.plan(key)
        return nmaps * (p.nalm * 16 + p.npix * 8)

    def launch(self, key, direction, datas, nmaps, slot):
        torch = self.torch
        p = self.plan(key)
        st = self.streams[slot]
        scr = self._grow(slot, p.workspace_bytes(sum(nmaps)))   # grows only beyond the warm-up size
        st.wait_stream(torch.cuda.current_stream(self.device))  # inputs were made on the caller's stream
        with torch.cuda.stream(st):
            x = datas[0] if len(datas) == 1 else torch.cat(datas, dim=0)
            y = p.alm2map_ws(x, scr, stream=st) if direction == ALM2MAP else p.map2alm_ws(x, scr, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, y, list(nmaps), datas, x, scr)

    def done(self, handle) -> bool:
        return handle[0].query()

    def results(self, handle):
        y, nmaps = handle[1], handle[2]
        outs, o = [], 0
        for n in nmaps:
            outs.append(y[o:o + n])
            o += n
        return outs


def poisson_trace(rate_hz: float, n: int, make_request: Callable[[int], Request], seed: int = 0):
    """n requests with exponential inter-arrival times of mean 1/rate_hz."""
    import numpy as np
    g = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    for i in range(n):
        t += float(g.exponential(1.0 / rate_hz))
        out.append((t, make_request(i)))
    return out
