"""Continuous-batching scheduler on a fake backend (CPU only): admission by
memory footprint, concurrency, per-system serialisation, eviction, and a
poisoned request that fails alone."""
import time

import numpy as np
import pytest

from paper_1303_4523_gb300.serving import Request, Server, SystemSpec, latency_stats


class FakeBackend:
    """Each request 'runs' for a fixed service time after launch."""

    def __init__(self, service=0.002, bytes_per_bead=100):
        self.service = service
        self.bpb = bytes_per_bead
        self.running = {}
        self.evicted = []
        self.launched = []

    def footprint(self, req):
        if req.system.params.get("poison"):
            raise ValueError("invalid parameters")
        return req.system.N * self.bpb

    def launch(self, key, req):
        if req.system.params.get("fail_launch"):
            raise RuntimeError("launch failed")
        assert key not in self.running, "two requests of one system in flight"
        self.running[key] = time.perf_counter() + self.service
        self.launched.append(req.rid)
        return (key, req)

    def done(self, h):
        return time.perf_counter() >= self.running[h[0]]

    def collect(self, h):
        key, req = h
        del self.running[key]
        return {"E": np.zeros(4), "beads_steps": req.system.N * (req.nsteps if req.kind == "dpd" else 1)}

    def evict(self, key):
        self.evicted.append(key)


def _sys(sid, N, **params):
    return SystemSpec(sid=sid, L=10.0, params=params, pos=np.zeros((N, 3)), q=np.zeros(N))


def test_all_served_and_concurrent():
    be = FakeBackend()
    srv = Server(be, budget_bytes=10**9, max_inflight=4)
    for k in range(12):
        srv.submit(Request(rid=k, kind="force", system=_sys(f"s{k}", 100), arrival=0.0))
    res = srv.run(realtime=False)
    assert [r.rid for r in res] == list(range(12)) and all(r.ok for r in res)
    assert srv.max_concurrent == 4
    st = latency_stats(res)
    assert st["n"] == 12 and st["p50_ms"] <= st["p99_ms"]


def test_budget_and_eviction():
    be = FakeBackend()
    srv = Server(be, budget_bytes=250 * 100, max_inflight=8)   # room for 250 beads
    for k in range(6):
        srv.submit(Request(rid=k, kind="force", system=_sys(f"s{k}", 100), arrival=0.0))
    res = srv.run(realtime=False)
    assert all(r.ok for r in res)
    assert srv.max_used <= 250 * 100 and srv.max_concurrent <= 2
    assert len(be.evicted) >= 4          # idle systems made room (LRU)


def test_requests_of_one_system_are_serialised():
    be = FakeBackend()
    srv = Server(be, budget_bytes=10**9, max_inflight=8)
    s = _sys("same", 100)
    for k in range(5):
        srv.submit(Request(rid=k, kind="dpd", system=s, arrival=0.0))
    res = srv.run(realtime=False)       # FakeBackend.launch asserts no overlap per key
    assert all(r.ok for r in res) and be.launched == list(range(5))


def test_poisoned_and_oversized_requests_fail_alone():
    be = FakeBackend()
    srv = Server(be, budget_bytes=1000 * 100, max_inflight=4)
    srv.submit(Request(rid=0, kind="force", system=_sys("a", 100), arrival=0.0))
    srv.submit(Request(rid=1, kind="force", system=_sys("bad", 100, poison=True), arrival=0.0))
    srv.submit(Request(rid=2, kind="force", system=_sys("huge", 5000), arrival=0.0))
    srv.submit(Request(rid=3, kind="force", system=_sys("boom", 100, fail_launch=True), arrival=0.0))
    srv.submit(Request(rid=4, kind="dpd", system=_sys("b", 100), arrival=0.0))
    res = {r.rid: r for r in srv.run(realtime=False)}
    assert res[0].ok and res[4].ok
    assert not res[1].ok and "invalid" in res[1].error
    assert not res[2].ok and "budget" in res[2].error
    assert not res[3].ok and "launch failed" in res[3].error


def test_arrivals_are_honoured():
    be = FakeBackend(service=0.001)
    srv = Server(be, budget_bytes=10**9, max_inflight=4)
    for k in range(4):
        srv.submit(Request(rid=k, kind="force", system=_sys(f"s{k}", 10), arrival=0.02 * k))
    t0 = time.perf_counter()
    res = srv.run(realtime=True)
    assert time.perf_counter() - t0 >= 0.06
    assert all(r.ok and r.latency < 0.05 for r in res)
