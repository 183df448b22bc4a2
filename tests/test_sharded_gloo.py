"""The m/ring-sharded transform (paper_1106_0159_gb300/sharded.py) on CPU ranks: the partition's
invariants, and a synthesis and an analysis run by two gloo ranks that exchange Delta with
point-to-point sends and receives.  The per-rank compute here is the oracle's separable stages
(the library needs a GPU); the result of the two ranks together must equal the oracle's whole
transform.  Unmeasured on hardware: this run has one GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import geometry
from paper_1106_0159_gb300 import inputs, sharded

NSIDE, L = 8, 16


class OracleStages:
    """One rank's four steps, from the oracle's separable forms."""

    def __init__(self, part, rank, geom, lmax):
        self.part, self.rank, self.geom, self.L = part, rank, geom, lmax
        self.ms = part.ms[rank]
        self.rings = part.rings[rank]

    def legendre_synth(self, alm):
        lv, mv = inputs.lm_arrays(self.L, self.part.mmax)
        mine = np.isin(mv, self.ms)
        out = []
        for a in alm:
            d = oracle.delta_synth(self.geom, np.where(mine, a, 0.0), self.L, self.part.mmax)
            out.append(d[:, self.ms])
        return np.stack(out)

    def ring_synth(self, d_rings):
        return np.stack([oracle.ring_synth(self.geom, d, self.part.mmax, self.rings) for d in d_rings])

    def ring_anal(self, pixels):
        off = geometry.ring_offsets(self.geom)
        out = []
        for px in pixels:
            full = np.zeros(int(off[-1]))
            o = 0
            for r in self.rings:
                n = int(off[r + 1] - off[r])
                full[off[r]:off[r + 1]] = px[o:o + n]
                o += n
            d = oracle.delta_anal(self.geom, full, np.arange(self.part.mmax + 1))  # [m][ring]
            out.append(d.T[self.rings])
        return np.stack(out)

    def legendre_anal(self, d_mine):
        out = []
        for d in d_mine:
            parts = oracle.legendre_anal(self.geom, np.ascontiguousarray(d.T), self.L, self.ms)
            a = np.zeros(oracle.nalm(self.L, self.part.mmax), dtype=np.complex128)
            for m, v in zip(self.ms, parts):
                i0 = oracle.alm_index(self.L, int(m), int(m))
                a[i0:i0 + len(v)] = v
            out.append(a)
        return np.stack(out)


class NumpyTorchExchange(sharded.TorchExchange):
    """The process-group transpose on numpy buffers (gloo sends torch CPU tensors)."""

    def exchange(self, send, recv_shapes, like):
        import torch
        tsend = {q: torch.from_numpy(np.ascontiguousarray(v)) for q, v in send.items()}
        recv = super().exchange(tsend, recv_shapes, torch.from_numpy(np.ascontiguousarray(like)))
        return {q: v.numpy() for q, v in recv.items()}


def test_partition_invariants():
    geom = geometry.healpix(16)
    for n in (1, 2, 3, 5):
        p = sharded.Partition(geom[0], geom[1], 40, n)
        ms = np.sort(np.concatenate(p.ms))
        assert np.array_equal(ms, np.arange(41))                       # every m once
        for r in range(n):                                             # min-max pairs stay together
            for m in p.ms[r]:
                assert (40 - m) in p.ms[r]
        rings = np.sort(np.concatenate(p.rings))
        assert np.array_equal(rings, np.arange(len(geom[0])))         # every ring once
        th = np.asarray(geom[1])
        for r in range(n):                                             # mirrors stay together
            own = set(p.rings[r].tolist())
            for i in own:
                mate = np.argmin(np.abs(th + th[i] - np.pi))
                assert int(mate) in own
        px = [int(np.sum(np.asarray(geom[0])[x])) for x in p.rings]
        assert max(px) - min(px) <= 2 * 4 * 16 + 2 * 64               # within a couple of slots
        # eq. msg_size: rank r sends R_q |M_r| values to q, R (mmax + 1) in all per map
        tot = sum(p.message_values(r, q) for r in range(n) for q in range(n))
        assert tot == len(geom[0]) * 41
        assert p.message_bytes(0, n - 1, nmaps=3) == 16 * 3 * len(p.rings[n - 1]) * len(p.ms[0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo")
    geom = geometry.healpix(NSIDE)
    part = sharded.Partition(geom[0], geom[1], L, world)
    st = OracleStages(part, rank, geom, L)
    ex = NumpyTorchExchange(rank, world)
    alm = inputs.gaussian_alm(L, L, seed=81, nmaps=2)
    pix = sharded.alm2map(part, rank, st, alm, ex)
    wm = inputs.white_map(geometry.npix(geom), seed=82, nmaps=2)
    off = geometry.ring_offsets(geom)
    mine = np.stack([np.concatenate([w[off[r]:off[r + 1]] for r in part.rings[rank]]) for w in wm])
    a = sharded.map2alm(part, rank, st, mine, ex)
    out.put((rank, pix, a))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_transform():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, pix, a = q.get(timeout=300)
        res[r] = (pix, a)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    geom = geometry.healpix(NSIDE)
    part = sharded.Partition(geom[0], geom[1], L, 2)
    off = geometry.ring_offsets(geom)
    alm = inputs.gaussian_alm(L, L, seed=81, nmaps=2)
    wm = inputs.white_map(geometry.npix(geom), seed=82, nmaps=2)
    for g in range(2):
        # synthesis: each rank's pixels are those rings of the whole map
        want = oracle.alm2map_rings(geom, alm[g], L, L)
        got = np.zeros_like(want)
        for r in range(2):
            o = 0
            for ring in part.rings[r]:
                n = int(off[ring + 1] - off[ring])
                got[off[ring]:off[ring + 1]] = res[r][0][g][o:o + n]
                o += n
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))
        # analysis: the ranks' a_lm (each its own m) add up to the whole analysis
        want = oracle.map2alm_rings(geom, wm[g], L, L)
        got = res[0][1][g] + res[1][1][g]
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))
