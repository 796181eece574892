"""Serving on the GPU: every request's result is the same alone and in a mix
of concurrently admitted requests (within the path's tolerance), work of
different systems overlaps, and a request with invalid parameters fails alone."""
import math

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _specs():
    from paper_1303_4523_gb300.serving import _spec_from
    out = [_spec_from(W.electrolyte(N, seed_offset=900 + k), f"e{k}") for k, N in
           enumerate([2000, 3000, 6000, 12000, 24000])]
    out.append(_spec_from(W.polyelectrolyte(L=8.0, n_chains=2, chain_len=20, seed_offset=901), "poly"))
    return out


def _requests(specs):
    from paper_1303_4523_gb300.serving import Request
    reqs = []
    rid = 0
    for s in specs[:5]:
        reqs.append(Request(rid=rid, kind="force", system=s, prec="fp32"))
        rid += 1
    reqs.append(Request(rid=rid, kind="force", system=specs[2], prec="fp64")); rid += 1
    reqs.append(Request(rid=rid, kind="dpd", system=specs[5], nsteps=3, prec="fp64")); rid += 1
    reqs.append(Request(rid=rid, kind="dpd", system=specs[0], nsteps=3, prec="fp64")); rid += 1
    reqs.append(Request(rid=rid, kind="dpd", system=specs[1], nsteps=3, prec="fp32")); rid += 1
    return reqs


def _rel(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def test_same_alone_and_in_mix():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300.serving import GpuBackend, Server
    specs = _specs()
    alone = {}
    for req in _requests(specs):
        be = GpuBackend()
        srv = Server(be, budget_bytes=8 << 30, max_inflight=1)
        srv.submit(req)
        (r,) = srv.run(realtime=False)
        assert r.ok, r.error
        alone[req.rid] = r
        srv.close()
    be = GpuBackend()
    srv = Server(be, budget_bytes=8 << 30, max_inflight=8)
    for req in _requests(specs):
        srv.submit(req)
    mix = {r.rid: r for r in srv.run(realtime=False)}
    srv.close()
    assert srv.max_concurrent > 1
    for req in _requests(specs):
        a, m = alone[req.rid], mix[req.rid]
        assert m.ok, m.error
        tolF = 1e-5 if req.prec == "fp32" else 1e-11
        assert _rel(m.F.astype(np.float64), a.F.astype(np.float64)) < tolF, req.rid
        if req.kind == "dpd":
            tolx = 1e-5 if req.prec == "fp32" else 1e-11
            assert np.abs(m.pos - a.pos).max() < tolx * req.system.L and m.step == a.step == req.nsteps
        # FP32 pair sums of alternating sign: the scale of the self term (as the parity tests)
        assert np.allclose(m.E[:4], a.E[:4], rtol=1e-6 if req.prec == "fp32" else 1e-11,
                           atol=1e-6 * abs(a.E[2]) if req.prec == "fp32" else 0.0)


def test_invalid_request_fails_alone():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300.serving import GpuBackend, Request, Server, SystemSpec
    specs = _specs()
    bad = SystemSpec(sid="bad", L=4.0, params=dict(alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, p=4),
                     pos=np.zeros((10, 3)), q=np.zeros(10))
    srv = Server(GpuBackend(), budget_bytes=4 << 30, max_inflight=4)
    srv.submit(Request(rid=0, kind="force", system=specs[0]))
    srv.submit(Request(rid=1, kind="force", system=bad))
    srv.submit(Request(rid=2, kind="force", system=specs[1]))
    res = {r.rid: r for r in srv.run(realtime=False)}
    srv.close()
    assert res[0].ok and res[2].ok and not res[1].ok and "invalid" in res[1].error
