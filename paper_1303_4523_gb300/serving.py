"""Continuous-batching server for ENUF-DPD requests.

Requests are ENUF force evaluations (one configuration of a system) or blocks
of DPD steps (Table 2) of a system whose state stays resident on the device.
They arrive over time; the scheduler admits each one as soon as an in-flight
slot and device memory (judged by the plan's HBM footprint plus the system's
state) are free, launches its work asynchronously on the system's own CUDA
stream, and collects it when its completion event has fired. Work of
different systems therefore overlaps on the GPU; requests of one system are
serialised. Idle resident systems are evicted least-recently-used when memory
is needed. A request that fails (bad parameters, out of memory) fails alone
with its status; the others are unaffected.

The scheduler talks to a backend with four calls (footprint, launch, done,
collect); GpuBackend drives libenuf.so through the binding, and tests use a
fake backend to check the scheduling on a CPU.
"""
from __future__ import annotations

import heapq
import math
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Any

import numpy as np


@dataclass
class SystemSpec:
    """One simulated system: box, ENUF parameters, bead arrays (host numpy)."""
    sid: str
    L: float
    params: dict                  # alpha, r_cut, beta, kappa, p (and optionally M, kmask, tile)
    pos: np.ndarray
    q: np.ndarray
    vel: np.ndarray | None = None
    types: np.ndarray | None = None
    bonds: np.ndarray | None = None
    dpd: dict | None = None       # a (ntypes x ntypes), gamma, sigma, dt, lambda_vv, K_bond, r0_bond, seed
    M: int = 0

    @property
    def N(self) -> int:
        return int(self.q.shape[0])


@dataclass
class Request:
    rid: int
    kind: str                     # "force" or "dpd"
    system: SystemSpec
    arrival: float = 0.0          # seconds after the start of the run
    nsteps: int = 10
    pos: np.ndarray | None = None  # force requests: configuration to evaluate (default: system.pos)
    prec: str = "fp32"


@dataclass
class Result:
    rid: int
    kind: str
    ok: bool
    error: str = ""
    latency: float = 0.0
    queued: float = 0.0
    F: np.ndarray | None = None
    E: np.ndarray | None = None
    pos: np.ndarray | None = None
    vel: np.ndarray | None = None
    step: int = 0
    beads_steps: int = 0


@dataclass(order=True)
class _Pending:
    arrival: float
    rid: int
    req: Request = field(compare=False)


class Server:
    """Admission, dispatch and collection of requests (continuous batching)."""

    def __init__(self, backend, budget_bytes: int, max_inflight: int = 8, poll_sleep: float = 5e-5):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.poll_sleep = poll_sleep
        self.pending: list[_Pending] = []
        self.inflight: dict[int, tuple[Request, Any, float]] = {}
        self.resident: "OrderedDict[str, int]" = OrderedDict()   # sid -> bytes, LRU order
        self.busy: set[str] = set()
        self.used = 0
        self.results: list[Result] = []
        self.max_used = 0
        self.max_concurrent = 0

    def submit(self, req: Request):
        heapq.heappush(self.pending, _Pending(req.arrival, req.rid, req))

    # -- memory -----------------------------------------------------------------
    def _key(self, req: Request) -> str:
        return f"{req.system.sid}/{req.kind}/{req.prec}"

    def _make_room(self, need: int) -> bool:
        while self.used + need > self.budget:
            victim = next((k for k in self.resident if k not in self.busy), None)
            if victim is None:
                return False
            self.used -= self.resident.pop(victim)
            self.backend.evict(victim)
        return True

    def _try_admit(self, req: Request, now: float) -> bool:
        key = self._key(req)
        if key in self.busy or len(self.inflight) >= self.max_inflight:
            return False
        need = 0
        if key not in self.resident:
            try:
                need = int(self.backend.footprint(req))
            except Exception as e:   # invalid request: fails alone
                self._finish(req, now, now, ok=False, error=str(e))
                return True
            if need > self.budget:
                self._finish(req, now, now, ok=False, error=f"needs {need} bytes > budget {self.budget}")
                return True
            if not self._make_room(need):
                return False
        try:
            handle = self.backend.launch(key, req)
        except Exception as e:
            if key in self.resident:
                self.used -= self.resident.pop(key)
            self.backend.evict(key)
            self._finish(req, now, now, ok=False, error=str(e))
            return True
        if key not in self.resident:
            self.resident[key] = need
            self.used += need
        self.resident.move_to_end(key)
        self.busy.add(key)
        self.inflight[req.rid] = (req, handle, now)
        self.max_used = max(self.max_used, self.used)
        self.max_concurrent = max(self.max_concurrent, len(self.inflight))
        return True

    def _finish(self, req, now, admitted, ok=True, error="", **kw):
        self.results.append(Result(rid=req.rid, kind=req.kind, ok=ok, error=error,
                                   latency=now - req.arrival, queued=admitted - req.arrival, **kw))

    # -- main loop ----------------------------------------------------------------
    def run(self, clock=time.perf_counter, realtime: bool = True):
        """Serve every submitted request; arrivals are honoured in real time
        (realtime=False admits each request as soon as possible)."""
        t0 = clock()
        while self.pending or self.inflight:
            now = clock() - t0
            progressed = False
            # admit in arrival order (FIFO: the head blocks the queue)
            while self.pending and (not realtime or self.pending[0].arrival <= now):
                head = self.pending[0]
                if not self._try_admit(head.req, now):
                    break
                heapq.heappop(self.pending)
                progressed = True
            # collect what finished
            for rid in list(self.inflight):
                req, handle, admitted = self.inflight[rid]
                if self.backend.done(handle):
                    key = self._key(req)
                    now = clock() - t0
                    try:
                        out = self.backend.collect(handle)
                        self._finish(req, now, admitted, ok=True, **out)
                    except Exception as e:
                        self._finish(req, now, admitted, ok=False, error=str(e))
                    del self.inflight[rid]
                    self.busy.discard(key)
                    progressed = True
            if not progressed:
                if self.pending and not self.inflight and realtime:
                    wait = self.pending[0].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                        continue
                time.sleep(self.poll_sleep)
        self.results.sort(key=lambda r: r.rid)
        return self.results

    def close(self):
        for key in list(self.resident):
            self.backend.evict(key)
        self.resident.clear()
        self.used = 0


def latency_stats(results: list[Result]) -> dict:
    lat = sorted(r.latency for r in results if r.ok)
    if not lat:
        return {"n": 0}
    def pct(p):
        return lat[min(len(lat) - 1, max(0, int(math.ceil(p * len(lat))) - 1))]
    return {"n": len(lat), "p50_ms": 1e3 * pct(0.50), "p99_ms": 1e3 * pct(0.99), "mean_ms": 1e3 * float(np.mean(lat)),
            "failed": sum(1 for r in results if not r.ok)}


class GpuBackend:
    """Runs requests through libenuf.so. One plan (and stream) per resident
    system key; force requests reuse the plan and its device buffers, DPD
    requests a resident DpdSystem. With a tune cache (autotune.TuneCache),
    systems that name no tile take the cached tile edge and FFT path of their
    shape when there is one; nothing is timed while serving."""

    def __init__(self, device: int = 0, tune_cache=None):
        import torch

        from paper_1303_4523_gb300 import enuf
        self.torch = torch
        self.enuf = enuf
        self.device = torch.device("cuda", device)
        self.sys: dict[str, dict] = {}
        self.tune_cache = tune_cache

    def _params(self, req: Request):
        s = req.system
        kw = dict(s.params)
        kw.setdefault("M", s.M)
        p = self.enuf.make_params(L=s.L, prec=req.prec, **kw)
        if self.tune_cache is not None and not kw.get("tile"):
            from paper_1303_4523_gb300 import autotune
            p = autotune.cached_params(p, int(np.count_nonzero(s.q)), cache=self.tune_cache)
        return p

    def footprint(self, req: Request) -> int:
        s = req.system
        esz = 4 if req.prec == "fp32" else 8
        plan_bytes = self.enuf.enuf_footprint(self._params(req), s.N)
        if req.kind == "force":
            return plan_bytes + s.N * 7 * esz
        ncells = int(math.floor(s.L / (1 + 1e-5))) ** 3
        return plan_bytes + s.N * (21 * esz + 16) + ncells * 16 + 4096

    def launch(self, key: str, req: Request):
        torch, enuf = self.torch, self.enuf
        s = req.system
        dt = torch.float32 if req.prec == "fp32" else torch.float64
        npd = np.float32 if req.prec == "fp32" else np.float64
        ent = self.sys.get(key)
        if ent is None:
            plan = enuf.Plan(self._params(req), s.N)
            ent = {"plan": plan}
            if req.kind == "force":
                ent["pos"] = torch.empty((s.N, 3), dtype=dt, device=self.device)
                ent["q"] = torch.tensor(np.asarray(s.q, npd), device=self.device)
                ent["F"] = torch.empty((s.N, 3), dtype=dt, device=self.device)
                ent["hF"] = torch.empty((s.N, 3), dtype=dt).pin_memory()
                torch.cuda.current_stream().synchronize()   # q uploaded before the plan's stream reads it
            else:
                d = s.dpd
                ent["sys"] = enuf.DpdSystem(plan, d["a"], d["gamma"], d["sigma"], d["dt"], s.pos, s.vel, s.types,
                                            s.q, s.bonds, lambda_vv=d.get("lambda_vv", 0.65),
                                            K_bond=d.get("K_bond", 0.0), r0_bond=d.get("r0_bond", 0.0),
                                            seed=d.get("seed", 0))
            self.sys[key] = ent
        plan = ent["plan"]
        st = plan.stream
        ev = torch.cuda.Event()
        if req.kind == "force":
            src = req.pos if req.pos is not None else s.pos
            hpos = torch.from_numpy(np.ascontiguousarray(src, npd)).pin_memory()
            with torch.cuda.stream(st):
                ent["pos"].copy_(hpos, non_blocking=True)
            plan.enqueue(ent["pos"], ent["q"], ent["F"])
            with torch.cuda.stream(st):
                ent["hF"].copy_(ent["F"], non_blocking=True)
            ev.record(st)
            return (key, req, ev, hpos)
        ent["sys"].step(req.nsteps)
        ent["sys"].copy_energies()   # a step keeps its energies on the device unless asked
        ev.record(st)
        return (key, req, ev, None)

    def done(self, handle) -> bool:
        return handle[2].query()

    def collect(self, handle) -> dict:
        key, req, ev, _ = handle
        ent = self.sys[key]
        E = ent["plan"].last_energies()
        if req.kind == "force":
            return {"F": ent["hF"].numpy().copy(), "E": E[:4], "beads_steps": req.system.N}
        pos, vel, F, step = ent["sys"].get_state()
        return {"pos": pos, "vel": vel, "F": F, "E": E, "step": step, "beads_steps": req.system.N * req.nsteps}

    def evict(self, key: str):
        ent = self.sys.pop(key, None)
        if ent is None:
            return
        if "sys" in ent:
            ent["sys"].close()
        ent["plan"].close()


def synthetic_load(n_requests: int, rate_hz: float, seed: int = 7, n_min: int = 1000, n_max: int = 1_000_000,
                   dpd_fraction: float = 0.3, big: int | None = 3_000_000, prec: str = "fp32",
                   n_systems: int = 24):
    """Poisson arrivals of force evaluations and 10-step DPD blocks on systems
    with N log-uniform in [n_min, n_max] at density 3 (10% charged +-1,
    lambda = 0.25, p = 4), plus one large system of `big` beads."""
    from paper_1303_4523_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    systems = []
    for k in range(n_systems):
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        systems.append(_spec_from(W.electrolyte(N, seed_offset=500 + k), f"load{seed}-s{k}"))
    if big:
        systems.append(_spec_from(W.electrolyte(big, seed_offset=499), f"load{seed}-big"))
    t = 0.0
    reqs = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        s = systems[int(rng.integers(len(systems)))]
        kind = "dpd" if rng.uniform() < dpd_fraction else "force"
        reqs.append(Request(rid=rid, kind=kind, system=s, arrival=t, nsteps=10, prec=prec))
    return reqs


def _spec_from(sysm, sid):
    from paper_1303_4523_gb300 import workloads as W
    dp = W.dpd_params(int(sysm.types.max()) + 1)
    return SystemSpec(sid=sid, L=sysm.L, params=dict(sysm.params), pos=sysm.pos, q=sysm.q, vel=sysm.vel,
                      types=sysm.types, bonds=sysm.bonds, dpd=dp, M=sysm.M)
