"""Replica bookkeeping for runs on several GPUs of one node.

The transforms do not shard across GPUs here: every rank (one process per
GPU, launched by torchrun) runs an independent replica of the workload on its
own maps.  The only cross-rank traffic is host-side bookkeeping around the
timed region: a barrier on both sides and the maximum of the per-rank
elapsed times, from which the whole-job throughput is computed.
"""
from __future__ import annotations

import os


class Replicas:
    def __init__(self, backend: str | None = None, device=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend is None:
                backend = "nccl"
            kw = {}
            if backend == "nccl" and device is not None:
                kw["device_id"] = device
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float, device=None) -> float:
        """Maximum of a per-rank float (elapsed ms) over all ranks."""
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def seed(self, base: int) -> int:
        """Distinct, reproducible input seed for this rank's replica."""
        return int(base) + 7919 * self.rank

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def job_throughput(world: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job units per second: every rank processed units_per_rank in at most ms_max."""
    return world * units_per_rank / (ms_max * 1e-3)
