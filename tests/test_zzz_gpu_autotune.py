"""The autotuner on the device: every legal launch shape it may pick (tile edge,
FFT path, radix schedule) gives the default plan's forces and energies to
rounding, and the tuned choice is one of them, measured and cached.

This file is named so that pytest collects it after the other GPU tests."""
import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import autotune, enuf
    return autotune, enuf


def _system(name):
    if name == "electrolyte_M16":
        s = W.electrolyte_small("bench")
        return dict(L=s.L, M=s.M, **s.params), s
    # n = 128: FP32 plans choose between the composite and the plain radix schedule
    s = W.electrolyte(2000, 20.0, n_charged=400, seed_offset=71)
    return dict(L=20.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=64, p=4), s


def _run(enuf, params, pos, q):
    plan = enuf.Plan(params, q.shape[0])
    F = torch.empty_like(pos)
    E, _ = plan.energy_forces(pos, q, F)
    info = plan.info
    radices = [info.fft_radix[i] for i in range(info.fft_stages)]
    two = info.fft_two_factor
    plan.close()
    return F.double().cpu().numpy(), E, info.tile, (two, radices)


@pytest.mark.parametrize("name,prec,tol", [("electrolyte_M16", "fp32", 1e-5), ("electrolyte_M16", "fp64", 1e-11),
                                           ("electrolyte_M64", "fp32", 1e-5)])
def test_every_candidate_matches_the_default_plan(mods, tmp_path, name, prec, tol):
    A, enuf = mods
    P, s = _system(name)
    params = enuf.make_params(prec=prec, **P)
    dt = torch.float32 if prec == "fp32" else torch.float64
    pos = torch.tensor(s.pos, dtype=dt, device="cuda")
    q = torch.tensor(s.q, dtype=dt, device="cuda")
    F0, E0, t0, rad0 = _run(enuf, params, pos, q)
    cands = A.candidates(params, s.N)
    assert {"tile": t0, "fft_path": 0, "fft_radix": 0} in cands
    for c in cands:
        F, E, t, rad = _run(enuf, A._copy(params, **c), pos, q)
        assert t == c["tile"]
        two, radices = rad
        if c["fft_radix"] == 1:
            assert not two and all(r in (2, 3, 4, 5, 8) for r in radices), rad
        elif c["fft_radix"] == 0:
            assert rad == rad0
        else:
            assert not two
        rel = np.sqrt(((F - F0) ** 2).sum() / (F0 ** 2).sum())
        assert rel <= 2 * tol, (c, rel)          # both within tol of the oracle
        assert abs(E[3] - E0[3]) <= 10 * tol * abs(E0[3]), (c, E, E0)

    cache = A.TuneCache(str(tmp_path / "tune.json"))
    r = A.tune(params, s.N, pos, q, cache=cache,
               measure=lambda p, n, a, b: A.time_on_device(p, n, a, b, reps=3, warmup=2))
    assert not r["cached"] and {k: r[k] for k in A.CHOICES} in cands
    assert len(r["timings"]) == len(cands) and all(t["ms"] > 0 for t in r["timings"])
    assert r["ms"] == min(t["ms"] for t in r["timings"])
    again = A.tune(params, s.N, pos, q, cache=A.TuneCache(cache.path))
    assert again["cached"] and again["tile"] == r["tile"]
    tp = A.tuned_params(params, s.N, pos, q, cache=A.TuneCache(cache.path))
    F, E, t, _ = _run(enuf, tp, pos, q)
    assert t == r["tile"] and np.sqrt(((F - F0) ** 2).sum() / (F0 ** 2).sum()) <= 2 * tol
