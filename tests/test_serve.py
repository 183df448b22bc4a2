"""Host logic of the continuous-batching server, with a fake backend and a manual clock (no GPU)."""
import numpy as np
import pytest

from paper_1106_0159_gb300 import serve
from paper_1106_0159_gb300.serve import ALM2MAP, MAP2ALM, Request, Server


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """A batch takes `cost_per_map * nmaps` seconds of clock; the 'transform' of a request is
    data * 2 + key[1] so that mixing up results between requests is visible."""

    def __init__(self, clock, cost_per_map=1.0, io_bytes_per_map=10, resident=0):
        self.clock = clock
        self.cost = cost_per_map
        self.io = io_bytes_per_map
        self.res = resident
        self.launches = []

    def memory_budget(self):
        return 10 ** 12

    def resident_bytes(self):
        return self.res

    def batch_bytes(self, key, direction, nmaps):
        return self.io * nmaps

    def launch(self, key, direction, datas, nmaps, slot):
        self.launches.append((key, direction, list(nmaps), slot, self.clock()))
        ready = self.clock() + self.cost * sum(nmaps)
        return (ready, [d * 2 + key[1] for d in datas])

    def done(self, handle):
        return self.clock() >= handle[0]

    def results(self, handle):
        return handle[1]


def settle(srv, clk, dt=1.0, limit=10000):
    """Advance the manual clock and poll until the server is idle."""
    for _ in range(limit):
        if srv.idle():
            return
        clk.t += dt
        srv.poll()
    raise AssertionError("server did not go idle")


def req(direction, nside, lmax, nmaps, fill=None, deadline=None):
    data = np.full((nmaps, 3), float(fill if fill is not None else nmaps))
    return Request(direction, lmax, nside, data, nmaps, deadline=deadline)


def test_batches_group_same_plan_and_direction_in_arrival_order():
    clk = Clock()
    be = FakeBackend(clk)
    srv = Server(be, max_batch_maps=8, nstreams=1, clock=clk)
    rs = [srv.submit(req(ALM2MAP, 32, 64, 3, fill=1)),
          srv.submit(req(MAP2ALM, 32, 64, 2, fill=2)),      # other direction: not in the batch
          srv.submit(req(ALM2MAP, 64, 128, 1, fill=3)),     # other plan: not in the batch
          srv.submit(req(ALM2MAP, 32, 64, 4, fill=4)),
          srv.submit(req(ALM2MAP, 32, 64, 2, fill=5))]      # would exceed 8 maps: next batch
    srv.poll()
    assert be.launches[0][:3] == ((32, 64), ALM2MAP, [3, 4])
    settle(srv, clk)
    keys = [(l[0], l[1], l[2]) for l in be.launches]
    assert keys == [((32, 64), ALM2MAP, [3, 4]), ((32, 64), MAP2ALM, [2]), ((64, 128), ALM2MAP, [1]),
                    ((32, 64), ALM2MAP, [2])]
    for r in rs:   # each request gets its own result back
        assert r.status == "done"
        np.testing.assert_array_equal(r.result, r.data * 2 + r.lmax)


def test_request_larger_than_batch_runs_alone():
    clk = Clock()
    be = FakeBackend(clk)
    srv = Server(be, max_batch_maps=4, nstreams=1, clock=clk)
    big = srv.submit(req(ALM2MAP, 32, 64, 9))
    small = srv.submit(req(ALM2MAP, 32, 64, 1))
    srv.poll()
    assert be.launches[0][2] == [9]
    settle(srv, clk)
    assert be.launches[1][2] == [1]
    assert big.status == small.status == "done"


def test_streams_bound_concurrency_and_requests_join_while_others_run():
    clk = Clock()
    be = FakeBackend(clk, cost_per_map=1.0)
    srv = Server(be, max_batch_maps=16, nstreams=2, clock=clk)
    a = srv.submit(req(ALM2MAP, 32, 64, 4))
    srv.poll()                       # a on slot 0
    b = srv.submit(req(MAP2ALM, 32, 64, 2))
    c = srv.submit(req(MAP2ALM, 32, 64, 2))
    srv.poll()                       # b+c together on slot 1 while a runs
    assert [l[3] for l in be.launches] == [0, 1] and be.launches[1][2] == [2, 2]
    d = srv.submit(req(ALM2MAP, 32, 64, 1))
    srv.poll()
    assert len(be.launches) == 2     # no free stream: d waits
    clk.t = 4.0                      # b+c (4 s) and a (4 s) finish
    srv.poll()
    assert a.status == b.status == c.status == "done"
    assert be.launches[2][2] == [1] and d.status == "running"
    clk.t = 5.0
    srv.poll()
    assert d.status == "done"
    assert a.latency == 4.0 and d.start == 4.0 and d.latency == 5.0


def test_memory_admission_waits_but_idle_server_admits():
    clk = Clock()
    be = FakeBackend(clk, io_bytes_per_map=10, resident=50)
    srv = Server(be, max_batch_maps=4, nstreams=4, memory_budget=100, clock=clk)
    a = srv.submit(req(ALM2MAP, 32, 64, 4))      # 40 bytes + 50 resident = 90: fits
    b = srv.submit(req(MAP2ALM, 32, 64, 2))      # +20 = 110 > 100: waits
    srv.poll()
    assert a.status == "running" and b.status == "pending"
    clk.t = 4.0
    srv.poll()
    assert a.status == "done" and b.status == "running"
    settle(srv, clk)
    huge = srv.submit(req(ALM2MAP, 32, 64, 4))   # over budget even alone
    be.res = 500
    srv.poll()
    assert huge.status == "running"              # nothing in flight: admitted anyway
    assert srv.bytes_in_flight == 40


def test_cancel_and_deadline():
    clk = Clock()
    be = FakeBackend(clk)
    srv = Server(be, max_batch_maps=4, nstreams=1, clock=clk)
    a = srv.submit(req(ALM2MAP, 32, 64, 4))
    srv.poll()
    b = srv.submit(req(ALM2MAP, 32, 64, 1))
    c = srv.submit(req(MAP2ALM, 32, 64, 1, deadline=2.0))
    assert srv.cancel(b) is True and b.status == "cancelled"
    assert srv.cancel(a) is False                # running: finishes, result dropped
    clk.t = 4.0
    srv.poll()                                   # c waited 4 s > 2 s: timed out
    assert c.status == "timeout" and a.status == "cancelled" and a.result is None
    assert srv.idle()
    assert sorted(r.rid for r in srv.dropped) == sorted([a.rid, b.rid, c.rid])
    assert srv.stats() == {"requests": 0}


def test_plain_mode_runs_one_request_per_call_in_order():
    clk = Clock()
    be = FakeBackend(clk)
    srv = Server(be, nstreams=1, batching=False, clock=clk)
    for n in (1, 2, 3):
        srv.submit(req(ALM2MAP, 32, 64, n))
    settle(srv, clk)
    assert [l[2] for l in be.launches] == [[1], [2], [3]]


def test_stats_percentiles():
    clk = Clock()
    be = FakeBackend(clk, cost_per_map=1.0)
    srv = Server(be, nstreams=1, batching=False, clock=clk)
    for _ in range(100):
        srv.submit(req(ALM2MAP, 32, 64, 1), arrival=0.0)
    srv.poll()                       # first request starts at t = 0
    for step in range(1, 101):
        clk.t = float(step)
        srv.poll()
    st = srv.stats()
    assert st["requests"] == 100 and st["maps"] == 100 and st["batches"] == 100
    assert st["p50_ms"] == pytest.approx(50500.0, abs=500.0)
    assert st["p99_ms"] == pytest.approx(99000.0, abs=1000.0)
    assert st["max_ms"] == 100000.0 and st["maps_per_s"] == pytest.approx(1.0)


def test_run_trace_submits_on_time():
    class Ticking(Clock):
        def __call__(self):
            self.t += 0.25
            return self.t

    clk = Ticking()
    be = FakeBackend(clk, cost_per_map=0.5)
    srv = Server(be, nstreams=1, clock=clk)
    trace = serve.poisson_trace(2.0, 20, lambda i: req(ALM2MAP if i % 2 else MAP2ALM, 32, 64, 1 + i % 3), seed=3)
    offs = [t for t, _ in trace]
    assert all(b > a for a, b in zip(offs, offs[1:]))
    srv.run_trace(trace)
    assert len(srv.completed) == 20
    for (t, r) in trace:
        assert r.start >= r.arrival and r.done > r.start
        np.testing.assert_array_equal(r.result, r.data * 2 + r.lmax)


def test_submit_rejects_bad_requests():
    srv = Server(FakeBackend(Clock()), clock=Clock())
    with pytest.raises(ValueError):
        srv.submit(req("sideways", 32, 64, 1))
    with pytest.raises(ValueError):
        srv.submit(Request(ALM2MAP, 64, 32, None, 0))
