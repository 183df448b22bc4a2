"""The multi-GPU replica bookkeeping, run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1106_0159_gb300.replicas import Replicas, job_throughput


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r = Replicas(backend="gloo")
    r.barrier()
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    mx = r.max_over_ranks(ms)
    out.put((rank, mx, r.seed(1000), job_throughput(r.world, 16, mx)))
    r.barrier()
    r.close()


def test_two_gloo_ranks_agree_on_max_time_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert res[0][2] != res[1][2]                      # distinct replica seeds
    assert res[0][3] == pytest.approx(2 * 16 / 0.150)  # whole-job maps/s


def test_single_process_needs_no_process_group():
    r = Replicas()
    assert r.world == 1 and r.dist is None
    assert r.max_over_ranks(3.5) == 3.5
    r.close()
