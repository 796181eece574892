"""GPU parity of the DPD step (Table 2) against the FP64 CPU oracle."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def enuf():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf as e
    return e


def _system(L=8.0, chains=3, f=0.5, valency=1):
    s = W.polyelectrolyte(L=L, n_chains=chains, chain_len=20, f=f, salt_fraction=0.1, valency=valency,
                          seed_offset=40)
    return s


def _prep(prec, s):
    cast = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if prec == "fp32" else (
        lambda a: np.asarray(a, np.float64))
    return cast(s.pos), cast(s.vel), cast(s.q)


def _make(enuf, prec, s, pos, vel, q, dp, pairs=0):   # pairs 0: the precision's automatic form
    P = dict(L=s.L, M=s.M, **s.params)
    plan = enuf.Plan(enuf.make_params(prec=prec, pairs=pairs, **P), s.N)
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], pos, vel, s.types, q, s.bonds,
                          lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"], seed=dp["seed"])
    Po = orc.EwaldParams(**P)
    Do = orc.DpdParams(**dp)
    return plan, sysm, Po, Do


def _rel(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def _bead_max(F, R):
    """Largest per-bead error |F_i - R_i| / max(|R_i|, rms_j |R_j|)."""
    rn = np.linalg.norm(R, axis=1)
    rms = math.sqrt((rn ** 2).mean())
    return float((np.linalg.norm(F - R, axis=1) / np.maximum(rn, rms)).max())


def _check_forces(F, R, tol):
    """Relative RMS below the path's bound, and no bead above 100x it."""
    F = np.asarray(F, np.float64)
    assert _rel(F, R) < tol, _rel(F, R)
    assert _bead_max(F, R) < 100 * tol, _bead_max(F, R)


@pytest.mark.parametrize("pairs", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_initial_force_parity(enuf, prec, tol, pairs):
    """Table 2 steps 3-5 at step 0: DPD C + D + R/sqrt(dt) + bonds + electrostatics
    (pairs = 1: the DPD and real-space pairs in two launches; 2: one launch)."""
    s = _system()
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, Po, Do = _make(enuf, prec, s, pos, vel, q, dp, pairs)
    _, _, F, step = sysm.get_state()
    Fr, Er = orc.total_forces(Po, Do, pos, vel, s.types, q, s.bonds, step=0)
    assert step == 0
    _check_forces(F, Fr, tol)
    sysm.close()
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_density4_force_parity(enuf, prec, tol):
    """The paper's density 4 (Table 1): the cell blocks shrink to 3^3 so their
    halos stay within the staging capacity; forces against the oracle."""
    s = W.polyelectrolyte(L=10.0, density=4.0, n_chains=2, chain_len=48, f=1.0, salt_fraction=0.05,
                          seed_offset=44)
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, Po, Do = _make(enuf, prec, s, pos, vel, q, dp)
    _, _, F, _ = sysm.get_state()
    Fr, _ = orc.total_forces(Po, Do, pos, vel, s.types, q, s.bonds, step=0)
    _check_forces(F, Fr, tol)
    sysm.step(2)
    sysm.close()
    plan.close()


@pytest.mark.parametrize("pairs", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_trajectory_parity(enuf, prec, pairs):
    """Three modified velocity-Verlet steps; positions, velocities, forces and
    energies against the oracle's Table 2 integrator."""
    s = _system(valency=2)
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, Po, Do = _make(enuf, prec, s, pos, vel, q, dp, pairs)
    F0, _ = orc.total_forces(Po, Do, pos, vel, s.types, q, s.bonds, step=0)
    pr, vr, Fr, st, Er = orc.dpd_run(Po, Do, pos, vel, F0, s.types, q, s.bonds, step=0, nsteps=3)
    E = sysm.step(3, want_energy=True)
    p, v, F, step = sysm.get_state()
    assert step == st == 3
    tp, tv, tF, tE = (1e-12, 1e-10, 1e-9, 1e-10) if prec == "fp64" else (1e-6, 2e-5, 2e-4, 1e-5)
    assert np.abs(p - pr).max() < tp * s.L
    assert _rel(v.astype(np.float64), vr) < tv
    assert _rel(F.astype(np.float64), Fr) < tF
    scale = max(abs(Er[0]), abs(Er[1]), abs(Er[2]))
    for k in range(4):
        assert abs(E[k] - Er[k]) < tE * scale, (k, E[:6], Er)
    assert abs(E[4] - Er[4]) < tE * abs(Er[4])
    assert abs(E[5] - Er[5]) < tE * max(abs(Er[5]), 1.0)
    assert abs(E[6] - 0.5 * (vr ** 2).sum()) < tE * 0.5 * (vr ** 2).sum()
    sysm.close()
    plan.close()


def test_restart_resumes_exactly(enuf):
    s = _system()
    dp = W.dpd_params(5)
    pos, vel, q = _prep("fp64", s)
    plan, sysm, _, _ = _make(enuf, "fp64", s, pos, vel, q, dp)
    sysm.step(4)
    pa, va, Fa, sa = sysm.get_state()
    sysm.set_state(pos, vel, None, 0)
    sysm.step(2)
    ck = sysm.get_state()
    sysm.set_state(ck[0], ck[1], ck[2], ck[3])
    sysm.step(2)
    pb, vb, Fb, sb = sysm.get_state()
    assert sa == sb == 4
    assert np.abs(pa - pb).max() < 1e-12 and np.abs(va - vb).max() < 1e-10
    sysm.close()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_host_equals_set_step_get(enuf, prec):
    """dpd_step_host (upload, steps, download, one synchronisation) gives the
    state and energies of set_state + step + get_state (to rounding: the bead
    order inside a binning tile follows shared-memory atomics)."""
    s = _system()
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, _, _ = _make(enuf, prec, s, pos, vel, q, dp)
    sysm.step(3)
    p0, v0, F0, st0 = sysm.get_state()
    Ea = sysm.step(2, want_energy=True)
    pa, va, Fa, sa = sysm.get_state()
    sysm.set_state(p0, v0, F0, st0)
    pb, vb, Fb = p0.copy(), v0.copy(), F0.copy()
    Eb = sysm.step_host(pb, vb, Fb, 2, want_energy=True)
    assert sysm.get_state()[3] == sa == st0 + 2
    rt = 1e-5 if prec == "fp32" else 1e-11
    assert np.allclose(pa, pb, rtol=rt, atol=rt) and np.allclose(va, vb, rtol=rt, atol=rt)
    assert _rel(Fb, Fa) < rt
    assert np.allclose(Ea, Eb, rtol=rt, atol=rt * np.abs(Ea).max())
    # NULL arrays keep the device copies and are not written back
    pc = pb.copy()
    sysm.step_host(pc, None, None, 1)
    pd, _, _, _ = sysm.get_state()
    assert np.array_equal(pc, pd)
    sysm.close()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_host_with_pinned_buffers(enuf, prec):
    """Pinned host tensors through dpd_step_host, one step at a time, match
    pageable arrays advanced two steps from the same state; other pinned
    tensors work the same way."""
    s = _system()
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, _, _ = _make(enuf, prec, s, pos, vel, q, dp)
    dt = torch.float32 if prec == "fp32" else torch.float64
    sysm.step(2)
    p0, v0, F0, st0 = sysm.get_state()
    # direct path (pageable arrays), two steps
    pa, va, Fa = p0.copy(), v0.copy(), F0.copy()
    sysm.step_host(pa, va, Fa, 2)
    # pinned tensors, two single steps from the same state
    sysm.set_state(p0, v0, F0, st0)
    tp, tv, tF = (torch.from_numpy(a.copy()).pin_memory() for a in (p0, v0, F0))
    E1 = sysm.step_host(tp, tv, tF, 1, want_energy=True)
    sysm.step_host(tp, tv, tF, 1)
    assert sysm.get_state()[3] == st0 + 2
    rt = 1e-5 if prec == "fp32" else 1e-11
    assert np.allclose(tp.numpy(), pa, rtol=rt, atol=rt) and np.allclose(tv.numpy(), va, rtol=rt, atol=rt)
    assert _rel(tF.numpy().astype(np.float64), Fa.astype(np.float64)) < rt
    assert np.isfinite(E1).all() and E1[6] > 0
    # other pinned arrays
    up, uv, uF = (t.clone().pin_memory() for t in (tp, tv, tF))
    sysm.step_host(up, uv, uF, 1)
    gp, _, _, st = sysm.get_state()
    assert st == st0 + 3 and np.array_equal(up.numpy(), gp)
    assert tp.dtype == dt
    sysm.close()
    plan.close()


def test_bad_inputs_are_rejected(enuf):
    s = _system()
    dp = W.dpd_params(5)
    P = dict(L=s.L, M=s.M, **s.params)
    plan = enuf.Plan(enuf.make_params(**P), s.N)
    bad_types = s.types.copy()
    bad_types[3] = 99
    with pytest.raises(enuf.EnufError):
        enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, bad_types, s.q, s.bonds)
    bad_bonds = s.bonds.copy()
    bad_bonds[0, 1] = s.N + 5
    with pytest.raises(enuf.EnufError):
        enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q, bad_bonds)
    plan.close()


def test_box_needs_three_cells_per_edge(enuf):
    """The staged DPD halo (block of B <= ncd - 2 cells plus one cell on each
    side) holds distinct cells only with ncd >= 3 cells of edge > 1: L = 3
    gives ncd = 2 (the edge rule keeps cells longer than 1 + 1e-5) and is
    rejected, L = 3.01 runs."""
    dp = W.dpd_params(5)
    rng = np.random.default_rng(11)
    n = 64
    for L, ok in [(3.0, False), (3.01, True)]:
        pos = rng.uniform(0.0, L, (n, 3))
        vel = rng.normal(0.0, 1.0, (n, 3))
        types = np.zeros(n, np.int32)
        q = np.zeros(n)
        plan = enuf.Plan(enuf.make_params(L=L, alpha=1.0, r_cut=1.4, beta=0.0, kappa=1.0, M=4, p=2), n)
        args = (plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], pos, vel, types, q, np.zeros((0, 2), np.int32))
        if ok:
            sysm = enuf.DpdSystem(*args)
            sysm.step(2)
            _, _, F, _ = sysm.get_state()
            assert np.all(np.isfinite(F))
            sysm.close()
        else:
            with pytest.raises(enuf.EnufError):
                enuf.DpdSystem(*args)
        plan.close()


@pytest.mark.parametrize("pairs", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_full_size_polyelectrolyte_sampled(enuf, prec, tol, pairs):
    """The bench workload (81000 beads, L = 30): initial ENUF-DPD force of 256
    sampled beads against the oracle bead by bead."""
    s = W.polyelectrolyte()
    dp = W.dpd_params(5)
    pos, vel, q = _prep(prec, s)
    plan, sysm, Po, Do = _make(enuf, prec, s, pos, vel, q, dp, pairs)
    _, _, F, _ = sysm.get_state()
    rng = np.random.default_rng(3)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(q)[0], 128, replace=False),
                                     rng.choice(np.nonzero(q == 0)[0], 128, replace=False),
                                     s.bonds[:8].ravel()]))
    sample = np.unique(sample)
    Fd, _ = orc.dpd_forces(Po, Do, pos, vel, s.types, s.bonds, step=0, sample=sample)
    Fe, _, _ = orc.electrostatics(Po, pos, q, recip="enuf", sample=sample)
    Fr = Fd + Fe
    _check_forces(F[sample], Fr, tol)
    sysm.close()
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_dense_blob_uses_both_block_paths(enuf, prec, tol):
    """A blob of 600 extra beads in a 2^3 corner region: every cell block whose
    halo holds it has more beads than the kernel stages in shared memory and
    takes the global-memory path, the rest stay staged; forces and the DPD
    energies still match the oracle."""
    s = _system()
    rng = np.random.default_rng(11)
    nb = 600
    pos = np.concatenate([s.pos, rng.uniform(1.0, 3.0, size=(nb, 3))])
    vel = np.concatenate([s.vel, rng.normal(0.0, 1.0, size=(nb, 3))])
    types = np.concatenate([s.types, np.zeros(nb, np.int32)]).astype(np.int32)
    qq = np.concatenate([s.q, np.zeros(nb)])
    cast = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if prec == "fp32" else np.asarray
    pos, vel, qq = cast(pos), cast(vel), cast(qq)
    # the busiest 6^3-cell halo (4^3 cell blocks of edge L/ncd) holds more than 896 beads
    ncd = int(np.floor(s.L / (1.0 + 1e-5)))
    assert len(pos) > 896 and nb > 896 - 216 * 3
    dp = W.dpd_params(5)
    P = dict(L=s.L, M=s.M, **s.params)
    plan = enuf.Plan(enuf.make_params(prec=prec, **P), len(pos))
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], pos, vel, types, qq, s.bonds,
                          lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"], seed=dp["seed"])
    Po = orc.EwaldParams(**P)
    Do = orc.DpdParams(**dp)
    _, _, F, _ = sysm.get_state()
    E = sysm.step(0, want_energy=True)
    Fr, Er = orc.total_forces(Po, Do, pos, vel, types, qq, s.bonds, step=0)
    assert ncd >= 3
    _check_forces(F, Fr, tol)
    assert abs(E[4] - Er[4]) < (1e-10 if prec == "fp64" else 1e-5) * abs(Er[4])
    assert abs(E[5] - Er[5]) < (1e-10 if prec == "fp64" else 1e-5) * max(abs(Er[5]), 1.0)
    sysm.close()
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 2e-3), ("fp32", 4e-3)])
def test_energy_is_conserved_without_thermostat(enuf, prec, tol):
    """With gamma = sigma = 0 the Table-2 integrator is velocity Verlet, and in
    gradient mode the reciprocal forces are the exact gradient of the NFFT
    energy; with the real-space and window errors made negligible (alpha r_c =
    4.5, p = 8, beta = 4) the total E_kin + E_c + E_bond + E_elec of the whole
    GPU step must stay flat: bounded fluctuation, no drift."""
    s = W.polyelectrolyte(L=8.0, n_chains=3, chain_len=20, f=0.5, salt_fraction=0.1, seed_offset=41)
    params = dict(s.params, alpha=1.5, p=8, beta=4.0)
    P = dict(L=s.L, M=16, deriv=1, **params)
    dp = W.dpd_params(5, gamma=0.0, sigma=0.0, dt=0.005)
    plan = enuf.Plan(enuf.make_params(prec=prec, **P), s.N)
    pos, vel, q = _prep(prec, s)
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], pos, vel, s.types, q, s.bonds,
                          lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"], seed=dp["seed"])
    H = []
    for _ in range(40):
        E = sysm.step(10, want_energy=True)
        H.append(E[3] + E[4] + E[5] + E[6])
    H = np.array(H)
    kin = E[6]
    assert np.all(np.isfinite(H))
    assert np.abs(H - H[0]).max() < tol * kin, (H.min(), H.max(), kin)
    assert abs(H[-10:].mean() - H[:10].mean()) < tol * kin
    sysm.close()
    plan.close()
