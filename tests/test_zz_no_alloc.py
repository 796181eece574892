"""The allocation-free spreading entry point (enuf_spread_noalloc).

Some callers may not allocate device memory (they run inside another
framework's memory pool, on a hot path where cudaMalloc is forbidden because
it can synchronise the device, or under a fixed memory budget). This entry
point gives them the spread grid of the ENUF path using only the caller's
arrays and the library's fixed 16 MiB device scratch. The test calls it
through the C ABI twice in a row and compares each result with the spread
grid of the regular, plan-based entry point.

This file is named so that pytest collects it after the plan-based tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_spread_matches_plan_grid(prec, tol):
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf

    s = W.electrolyte_small("bench")
    params = enuf.make_params(prec=prec, L=s.L, M=s.M, **s.params)
    dt = torch.float32 if prec == "fp32" else torch.float64
    pos = torch.tensor(s.pos, dtype=dt, device="cuda")
    q = torch.tensor(s.q, dtype=dt, device="cuda")

    plan = enuf.Plan(params, s.N)
    F = torch.empty_like(pos)
    plan.energy_forces(pos, q, F)
    ref = plan.debug_buffer(enuf.ENUF_BUF_GRID).astype(np.float64)
    n = plan.info.n
    plan.close()

    stream = torch.cuda.current_stream()
    for call in range(2):
        grid = torch.full((n, n, n), float("nan"), dtype=dt, device="cuda")
        st = enuf.lib.enuf_spread_noalloc(C.byref(params), s.N, pos.data_ptr(), q.data_ptr(),
                                          grid.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        g = grid.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - ref).max() <= tol * np.abs(ref).max(), call


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf

    params = enuf.make_params(L=60.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=96, p=4)
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    # the size check comes before any device work, so the small buffers are never read
    st = enuf.lib.enuf_spread_noalloc(C.byref(params), 5_000_000, x.data_ptr(), x.data_ptr(), x.data_ptr(), None)
    assert st == 1
