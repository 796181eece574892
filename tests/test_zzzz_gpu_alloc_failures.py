"""Out-of-memory paths, by failure injection on the host: the library's next
device allocations report out-of-memory without calling the allocator
(enuf_debug_fail_allocs), so no GPU is exhausted or faulted. Each failing call
returns ENUF_ERR_OOM alone and frees what it held; the next call succeeds and
gives the same result as before.

This file is named so that pytest collects it after the other GPU tests."""
import math

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def enuf():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf as E
    return E


@pytest.fixture(autouse=True)
def _no_injection_left(enuf):
    yield
    enuf.debug_fail_allocs(0)


def _rel(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def _setup(enuf):
    s = W.electrolyte_small("bench")
    params = enuf.make_params(prec="fp64", L=s.L, M=s.M, **s.params)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    q = torch.tensor(s.q, dtype=torch.float64, device="cuda")
    return s, params, pos, q


def _forces(plan, pos, q):
    F = torch.empty_like(pos)
    E, _ = plan.energy_forces(pos, q, F)
    return F.cpu().numpy(), E


def test_plan_and_staging_allocations(enuf):
    s, params, pos, q = _setup(enuf)
    plan0 = enuf.Plan(params, s.N)
    F0, E0 = _forces(plan0, pos, q)
    # the host-only shape query describes the plan that was built
    shape, info = enuf.plan_shape(params, s.N), plan0.info
    for f in ("M", "n", "n_c", "tile", "n_tiles", "n_max", "fft_kernels", "device_bytes", "fft_stages"):
        assert getattr(shape, f) == getattr(info, f), f
    assert list(shape.fft_radix) == list(info.fft_radix)
    enuf.debug_fail_allocs(1)
    with pytest.raises(enuf.EnufError) as e:
        enuf.Plan(params, s.N)
    assert e.value.status == enuf.ENUF_ERR_OOM
    plan = enuf.Plan(params, s.N)                       # the injection is used up
    F, E = _forces(plan, pos, q)
    assert _rel(F, F0) < 1e-12 and np.allclose(E, E0, rtol=1e-12)
    # the host-buffer entry point allocates its staging on first use
    Fh = np.empty((s.N, 3))
    enuf.debug_fail_allocs(1)
    with pytest.raises(enuf.EnufError) as e:
        plan.energy_forces_host(s.pos, s.q, Fh)
    assert e.value.status == enuf.ENUF_ERR_OOM
    Eh, _ = plan.energy_forces_host(s.pos, s.q, Fh)
    assert _rel(Fh, F0) < 1e-12 and np.allclose(Eh, E0, rtol=1e-12)
    # the plan that existed before the injection is untouched
    F1, _ = _forces(plan0, pos, q)
    assert _rel(F1, F0) < 1e-12
    plan.close()
    plan0.close()


def test_dpd_system_allocation(enuf):
    s = W.polyelectrolyte(L=8.0, n_chains=2, chain_len=20, seed_offset=931)
    params = enuf.make_params(prec="fp64", L=s.L, M=s.M, **s.params)
    plan = enuf.Plan(params, s.N)
    dp = W.dpd_params(int(s.types.max()) + 1)
    args = (plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q, s.bonds)
    kw = dict(lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"], seed=dp["seed"])
    ref = enuf.DpdSystem(*args, **kw)
    ref.step(3)
    p_ref, v_ref, _, _ = ref.get_state()
    ref.close()
    enuf.debug_fail_allocs(1)
    with pytest.raises(enuf.EnufError) as e:
        enuf.DpdSystem(*args, **kw)
    assert e.value.status == enuf.ENUF_ERR_OOM
    sysm = enuf.DpdSystem(*args, **kw)
    sysm.step(3)
    p, v, _, step = sysm.get_state()
    assert step == 3
    assert np.abs(p - p_ref).max() < 1e-9 * s.L and np.abs(v - v_ref).max() < 1e-9
    sysm.close()
    plan.close()


def test_batch_allocation(enuf):
    systems = [W.electrolyte(N, seed_offset=940 + k) for k, N in enumerate([2000, 3000, 4000])]
    params = [enuf.make_params(prec="fp64", L=s.L, M=s.M, **s.params) for s in systems]
    pos = [torch.tensor(s.pos, dtype=torch.float64, device="cuda") for s in systems]
    q = [torch.tensor(s.q, dtype=torch.float64, device="cuda") for s in systems]
    F = [torch.empty_like(p) for p in pos]
    enuf.debug_fail_allocs(1, after=1)                  # the second system's plan fails
    with pytest.raises(enuf.EnufError) as e:
        enuf.Batch(params, [s.N for s in systems])
    assert e.value.status == enuf.ENUF_ERR_OOM        # and the first one's is freed
    b = enuf.Batch(params, [s.N for s in systems])
    E = b.energy_forces(pos, q, F)
    b.close()
    for k, s in enumerate(systems):
        plan = enuf.Plan(params[k], s.N)
        Fk, Ek = _forces(plan, pos[k], q[k])
        plan.close()
        assert _rel(F[k].cpu().numpy(), Fk) < 1e-12
        assert np.allclose(np.asarray(E)[k][:4], Ek[:4], rtol=1e-12)


def test_batch_sequence_table_allocation(enuf):
    """FP32 batch run as one launch sequence: after its three plans, the
    allocation of the batch's argument tables fails; nothing is kept, and the
    next batch works."""
    systems = [W.electrolyte(N, seed_offset=960 + k) for k, N in enumerate([2000, 3000, 4000])]
    params = [enuf.make_params(prec="fp32", L=s.L, M=s.M, **s.params) for s in systems]
    pos = [torch.tensor(s.pos, dtype=torch.float32, device="cuda") for s in systems]
    q = [torch.tensor(s.q, dtype=torch.float32, device="cuda") for s in systems]
    F = [torch.empty_like(p) for p in pos]
    enuf.debug_fail_allocs(1, after=3)                  # the tables, after three plans
    with pytest.raises(enuf.EnufError) as e:
        enuf.Batch(params, [s.N for s in systems])
    assert e.value.status == enuf.ENUF_ERR_OOM
    b = enuf.Batch(params, [s.N for s in systems])
    assert b.mode() == 1
    E = b.energy_forces(pos, q, F)
    b.close()
    for k, s in enumerate(systems):
        plan = enuf.Plan(params[k], s.N)
        Fk, Ek = _forces(plan, pos[k], q[k])
        plan.close()
        assert _rel(F[k].cpu().numpy().astype(np.float64), Fk.astype(np.float64)) < 1e-6
        # FP32 pair sums of alternating sign: the scale of the self term (as the parity tests)
        assert np.allclose(np.asarray(E)[k][:4], Ek[:4], rtol=1e-6, atol=1e-6 * abs(Ek[2]))


def test_serving_request_fails_alone(enuf):
    from paper_1303_4523_gb300.serving import GpuBackend, Request, Server, _spec_from
    specs = [_spec_from(W.electrolyte(N, seed_offset=950 + k), f"s{k}") for k, N in enumerate([2000, 3000, 4000])]
    srv = Server(GpuBackend(), budget_bytes=4 << 30, max_inflight=1)
    for k, sp in enumerate(specs):
        srv.submit(Request(rid=k, kind="force", system=sp, prec="fp64"))
    enuf.debug_fail_allocs(1)                           # the first admitted request's plan
    res = {r.rid: r for r in srv.run(realtime=False)}
    srv.close()
    assert not res[0].ok and "out of device memory" in res[0].error
    assert res[1].ok and res[2].ok
