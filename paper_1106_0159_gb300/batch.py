"""A fixed batch of transforms (several plans, band limits, directions and map counts) run as
one CUDA graph.

Two forms.  PersistentBatch (plain FP64 plans): every transform of one direction is one library
batch (sht_batch_*): one persistent launch per stage whose CTAs take (transform, map group, m,
slot block) tiles of all plans from one device queue, longest l-range first, and (transform, ring
pair, map) DFT units longest first; the alm2map batch and the map2alm batch run on two streams
inside one graph, so the ring stage of one direction overlaps the Legendre stage of the other.
GraphBatch (any mode): one library call per job, as below.

Each job is one library call (sht_alm2map or sht_map2alm) with device buffers that stay put.
Jobs of one plan run in order on one stream (a plan's scratch serves one stream); the plans are
spread over a few streams that fork from and join the capture stream, so independent plans
overlap on the GPU.  capture() reserves every plan's scratch for its largest job and runs each
job once eagerly (kernels loaded, nothing left to allocate), then records the whole batch;
replay() launches it with one host call.  Inputs can be rewritten in place between replays.

The transforms run in the CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import dataclasses
from typing import Any, Dict, List, Optional

ALM2MAP, MAP2ALM = "alm2map", "map2alm"


@dataclasses.dataclass(eq=False)
class Job:
    plan: Any
    direction: str     # ALM2MAP or MAP2ALM
    src: Any           # [nmaps, nalm] complex128 or [nmaps, npix] float64, on the device
    dst: Any           # the output, preallocated

    @property
    def nmaps(self) -> int:
        return int(self.src.shape[0])


def assign_streams(jobs: List[Job], nstreams: int) -> List[List[Job]]:
    """Group jobs by plan (order kept within a plan) and deal the plans over `nstreams` streams,
    largest total work first onto the least-loaded stream (work ~ maps x lmax^3)."""
    by_plan: Dict[int, List[Job]] = {}
    order: List[int] = []
    for j in jobs:
        k = id(j.plan)
        if k not in by_plan:
            by_plan[k] = []
            order.append(k)
        by_plan[k].append(j)

    def work(js):
        return sum(j.nmaps for j in js) * float(js[0].plan.lmax) ** 3

    lanes: List[List[Job]] = [[] for _ in range(max(1, nstreams))]
    load = [0.0] * len(lanes)
    for k in sorted(order, key=lambda k: -work(by_plan[k])):
        i = min(range(len(lanes)), key=lambda i: load[i])
        lanes[i].extend(by_plan[k])
        load[i] += work(by_plan[k])
    return [ln for ln in lanes if ln]


class GraphBatch:
    def __init__(self, jobs: List[Job], nstreams: int = 2):
        for j in jobs:
            if j.direction not in (ALM2MAP, MAP2ALM):
                raise ValueError("unknown direction %r" % (j.direction,))
        self.jobs = list(jobs)
        self.lanes = assign_streams(self.jobs, nstreams)
        self.graph = None

    @staticmethod
    def _call(job: Job, stream):
        if job.direction == ALM2MAP:
            job.plan.alm2map(job.src, out=job.dst, stream=stream)
        else:
            job.plan.map2alm(job.src, out=job.dst, stream=stream)

    def run_eager(self, streams=None):
        """The same calls without a graph, on the given streams (default: the current stream)."""
        import torch
        cur = torch.cuda.current_stream()
        for i, lane in enumerate(self.lanes):
            st = streams[i] if streams else cur
            for job in lane:
                self._call(job, st)

    def capture(self):
        import torch
        most: Dict[int, int] = {}
        for j in self.jobs:
            most[id(j.plan)] = max(most.get(id(j.plan), 0), j.nmaps)
        for j in self.jobs:
            j.plan.reserve(most[id(j.plan)])
        self.run_eager()
        torch.cuda.synchronize()
        self.streams = [torch.cuda.Stream() for _ in self.lanes]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.streams[0]):
            s0 = self.streams[0]
            for st in self.streams[1:]:
                st.wait_stream(s0)
            for lane, st in zip(self.lanes, self.streams):
                for job in lane:
                    self._call(job, st)
            for st in self.streams[1:]:
                s0.wait_stream(st)
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()


class PersistentBatch:
    """All jobs of one direction in one sht batch (plain FP64 plans); the two directions on two
    streams of one CUDA graph.  Same interface as GraphBatch."""

    def __init__(self, jobs: List[Job], nstreams: int = 2):
        from . import sht
        self.jobs = list(jobs)
        self.batches = []
        for d, code in ((ALM2MAP, sht.BATCH_ALM2MAP), (MAP2ALM, sht.BATCH_MAP2ALM)):
            js = [j for j in self.jobs if j.direction == d]
            if js:
                self.batches.append((d, sht.Batch(code, [(j.plan, j.src, j.dst) for j in js])))
        for j in self.jobs:
            if j.direction not in (ALM2MAP, MAP2ALM):
                raise ValueError("unknown direction %r" % (j.direction,))
        self.nstreams = max(1, min(nstreams, len(self.batches)))
        self.graph = None
        self.streams = None

    def run_eager(self, streams=None):
        import torch
        cur = torch.cuda.current_stream()
        for i, (_, b) in enumerate(self.batches):
            st = streams[i % len(streams)] if streams else cur
            b.run(stream=st)

    def capture(self):
        import torch
        self.run_eager()
        torch.cuda.synchronize()
        self.streams = [torch.cuda.Stream() for _ in range(self.nstreams)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.streams[0]):
            s0 = self.streams[0]
            for st in self.streams[1:]:
                st.wait_stream(s0)
            for i, (_, b) in enumerate(self.batches):
                b.run(stream=self.streams[i % self.nstreams])
            for st in self.streams[1:]:
                s0.wait_stream(st)
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def close(self):
        for _, b in self.batches:
            b.close()
        self.batches = []
