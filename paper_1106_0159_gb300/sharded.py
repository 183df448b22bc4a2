"""One transform sharded over several GPUs by m and by rings, with one exchange of Delta.

This is the distribution of the paper's Section 4.1 (Algorithm 3): the Legendre step of rank r
covers its own set of m and every ring, the ring step its own rings and every m, and between the
two the Delta_m(ring) slab is transposed once, every rank sending rank q the rows of q's rings
for r's m.  Section 4.1's message estimate (eq. msg_size) is the size of that transpose: rank r
sends sum over q of nmaps |R_q| |M_r| complex values, R (mmax+1) / n per rank in total.

Ownership:
  - m: the min-max pairs (m, mmax - m) of Section 4.2.1 (load balance: the l-range of a pair is
    always mmax + 2 long) are dealt to the ranks round robin, so every rank's Legendre work is
    within one pair of the others';
  - rings: ring slots (a ring and its mirror, which share one DFT and one recurrence) in
    colatitude order, cut into contiguous groups of nearly equal pixel count.

The exchange is a set of point-to-point sends and receives, posted together
(`torch.distributed.batch_isend_irecv`: NCCL runs them as one grouped call; gloo on CPU ranks).
No multicast or collective other than that is used.  On GPUs the per-rank compute is the
library's own stages (`LibraryStages`: an m-list plan over every ring for the Legendre step and a
plan over the rank's rings for the ring step); any object with the same four methods can stand in
for it.  A `LoopbackExchange` runs every rank in one process (a transpose by copies), which lets
one GPU check the sharded path against the plain transforms.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- partition

class Partition:
    """Which rank owns which m and which rings."""

    def __init__(self, nphi, theta, mmax: int, nranks: int):
        self.nranks = int(nranks)
        self.mmax = int(mmax)
        self.nrings = len(nphi)
        nphi = np.asarray(nphi, dtype=np.int64)
        theta = np.asarray(theta, dtype=np.float64)
        # m: min-max pairs dealt round robin
        pairs = [(m, mmax - m) for m in range((mmax + 2) // 2)]
        self.ms = [[] for _ in range(self.nranks)]
        for k, (a, b) in enumerate(pairs):
            r = k % self.nranks
            self.ms[r].append(a)
            if b != a:
                self.ms[r].append(b)
        self.ms = [np.array(sorted(x), dtype=np.int64) for x in self.ms]
        # rings: slots = (a ring, its mirror), found as in the plan: rings sorted by colatitude,
        # paired from both ends when their colatitudes add to pi
        idx = np.argsort(theta, kind="stable")
        slots, i, j = [], 0, self.nrings - 1
        while i <= j:
            a, b = int(idx[i]), int(idx[j])
            if i == j:
                slots.append([a])
                break
            t = theta[a] + theta[b]
            if abs(t - np.pi) <= 4e-15:
                slots.append([a, b])
                i += 1
                j -= 1
            elif t < np.pi:
                slots.append([a])
                i += 1
            else:
                slots.append([b])
                j -= 1
        slots.sort(key=lambda sl: min(min(theta[r], np.pi - theta[r]) for r in sl))
        weight = np.array([sum(int(nphi[r]) for r in s) for s in slots], dtype=np.float64)
        cum = np.cumsum(weight)
        cuts = [int(np.searchsorted(cum, cum[-1] * (k + 1) / self.nranks - 1e-9)) + 1 for k in range(self.nranks)]
        self.rings, lo = [], 0
        for k in range(self.nranks):
            hi = len(slots) if k == self.nranks - 1 else max(lo, min(cuts[k], len(slots)))
            self.rings.append(np.array(sorted(r for s in slots[lo:hi] for r in s), dtype=np.int64))
            lo = hi

    def message_values(self, src: int, dst: int, nmaps: int = 1) -> int:
        """Complex values rank src sends rank dst in one exchange (eq. msg_size per pair)."""
        return int(nmaps) * len(self.rings[dst]) * len(self.ms[src])

    def message_bytes(self, src: int, dst: int, nmaps: int = 1) -> int:
        return 16 * self.message_values(src, dst, nmaps)


# ---------------------------------------------------------------- the transpose

def synth_sendbufs(part: Partition, rank: int, d_mine):
    """Synthesis: d_mine [nmaps][nrings][|M_rank|] -> {q: rows of q's rings}."""
    return {q: d_mine[:, part.rings[q], :] for q in range(part.nranks)}


def synth_assemble(part: Partition, rank: int, recv, like):
    """Synthesis: {r: [nmaps][|R_rank|][|M_r|]} -> Delta of this rank's rings, every m."""
    nmaps = next(iter(recv.values())).shape[0]
    out = _zeros(like, (nmaps, len(part.rings[rank]), part.mmax + 1))
    for r, buf in recv.items():
        out[:, :, part.ms[r]] = buf
    return out


def anal_sendbufs(part: Partition, rank: int, d_rings):
    """Analysis: Delta of this rank's rings [nmaps][|R_rank|][mmax+1] -> {r: r's m columns}."""
    return {r: d_rings[:, :, part.ms[r]] for r in range(part.nranks)}


def anal_assemble(part: Partition, rank: int, recv, like):
    """Analysis: {q: [nmaps][|R_q|][|M_rank|]} -> [nmaps][nrings][|M_rank|]."""
    nmaps = next(iter(recv.values())).shape[0]
    out = _zeros(like, (nmaps, part.nrings, len(part.ms[rank])))
    for q, buf in recv.items():
        out[:, part.rings[q], :] = buf
    return out


def _zeros(like, shape):
    if isinstance(like, np.ndarray):
        return np.zeros(shape, dtype=like.dtype)
    import torch
    return torch.zeros(shape, dtype=like.dtype, device=like.device)


class TorchExchange:
    """The transpose between processes: every rank posts its sends and receives together."""

    def __init__(self, rank: int, world: int):
        import torch.distributed as dist
        self.dist, self.rank, self.world = dist, rank, world

    def exchange(self, send, recv_shapes, like):
        import torch
        recv, ops = {}, []
        for q in range(self.world):
            if q == self.rank:
                recv[q] = send[q].clone()
                continue
            recv[q] = torch.empty(recv_shapes[q], dtype=like.dtype, device=like.device)
            ops.append(self.dist.P2POp(self.dist.isend, send[q].contiguous(), q))
            ops.append(self.dist.P2POp(self.dist.irecv, recv[q], q))
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        return recv


class LoopbackExchange:
    """Every rank in one process: the transpose is a set of copies (no process group)."""

    @staticmethod
    def exchange_all(sends):
        n = len(sends)
        return [{r: _copy(sends[r][q]) for r in range(n)} for q in range(n)]


def _copy(t):
    return t.copy() if isinstance(t, np.ndarray) else t.clone()


# ---------------------------------------------------------------- one rank's steps

def alm2map(part: Partition, rank: int, stages, alm, exch):
    """This rank's part of a sharded synthesis: alm (the full m-major layout; only this rank's m
    are read) -> pixels of this rank's rings [nmaps][npix_rank], ring order of part.rings[rank]."""
    d_mine = stages.legendre_synth(alm)                      # [nmaps][nrings][|M_rank|]
    send = synth_sendbufs(part, rank, d_mine)
    shapes = {r: (d_mine.shape[0], len(part.rings[rank]), len(part.ms[r])) for r in range(part.nranks)}
    recv = exch.exchange(send, shapes, d_mine)
    return stages.ring_synth(synth_assemble(part, rank, recv, d_mine))


def map2alm(part: Partition, rank: int, stages, pixels, exch):
    """This rank's part of a sharded analysis: pixels of this rank's rings -> a_lm in the full
    layout with this rank's m filled (zero elsewhere)."""
    d_rings = stages.ring_anal(pixels)                       # [nmaps][|R_rank|][mmax+1]
    send = anal_sendbufs(part, rank, d_rings)
    shapes = {q: (d_rings.shape[0], len(part.rings[q]), len(part.ms[rank])) for q in range(part.nranks)}
    recv = exch.exchange(send, shapes, d_rings)
    return stages.legendre_anal(anal_assemble(part, rank, recv, d_rings))


def alm2map_loopback(part: Partition, stages_per_rank, alm):
    """Every rank of a sharded synthesis in one process; returns each rank's pixels."""
    mine = [st.legendre_synth(alm) for st in stages_per_rank]
    sends = [synth_sendbufs(part, r, mine[r]) for r in range(part.nranks)]
    recvs = LoopbackExchange.exchange_all(sends)
    return [st.ring_synth(synth_assemble(part, q, recvs[q], mine[q])) for q, st in enumerate(stages_per_rank)]


def map2alm_loopback(part: Partition, stages_per_rank, pixels_per_rank):
    """Every rank of a sharded analysis in one process; returns each rank's a_lm."""
    rings = [st.ring_anal(px) for st, px in zip(stages_per_rank, pixels_per_rank)]
    sends = [anal_sendbufs(part, q, rings[q]) for q in range(part.nranks)]
    recvs = LoopbackExchange.exchange_all(sends)
    return [st.legendre_anal(anal_assemble(part, r, recvs[r], rings[r])) for r, st in enumerate(stages_per_rank)]


# ---------------------------------------------------------------- the library's stages on one GPU

class LibraryStages:
    """A rank's compute on its GPU through the C ABI (FP64 Legendre steps with an m list)."""

    def __init__(self, part: Partition, rank: int, geom, lmax: int, grid: int = 0):
        from . import sht
        nphi, theta, phi0, w = [np.asarray(x) for x in geom]
        self.part, self.rank = part, rank
        self.all = sht.Plan(geom, lmax, part.mmax, grid=grid)      # every ring, this rank's m
        self.all.set_mlist(part.ms[rank])
        r = part.rings[rank]
        self.own = sht.Plan((nphi[r], theta[r], phi0[r], w[r]), lmax, part.mmax)   # this rank's rings
        import torch
        self._cols = torch.as_tensor(part.ms[rank], device="cuda")

    def legendre_synth(self, alm):
        return self.all.legendre_synth(alm).index_select(2, self._cols)

    def ring_synth(self, d_rings):
        return self.own.ring_synth(d_rings.contiguous())

    def ring_anal(self, pixels):
        return self.own.ring_anal(pixels)

    def legendre_anal(self, d_mine):
        import torch
        full = torch.zeros((d_mine.shape[0], self.part.nrings, self.part.mmax + 1), dtype=d_mine.dtype,
                           device=d_mine.device)
        full[:, :, self._cols] = d_mine
        return self.all.legendre_anal(full)

    def close(self):
        self.all.close()
        self.own.close()
