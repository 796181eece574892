"""Pins of the oracle's DPD forces, random numbers and integrator (CPU only)."""
import math
import os

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W


def _box(n=300, L=5.0, seed=4):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, (n, 3))
    vel = rng.normal(0, 1, (n, 3))
    return pos, vel, np.zeros(n, dtype=np.int32), L


def _P(orc, L):
    return orc.EwaldParams(L=L, alpha=1.0, r_cut=min(3.0, L / 2), beta=4.0, kappa=1.0, M=16, p=4)


def test_theta_statistics(orc):
    """Eq. 5: theta_ij has zero mean and unit variance, and is symmetric in i, j."""
    n = 20000
    th = np.array([orc.theta(1303, 7, i, i + 1 + (i % 13)) for i in range(n)])
    assert abs(th.mean()) < 4.0 / math.sqrt(n)
    assert abs(th.var() - 1.0) < 0.03
    assert th.min() >= -math.sqrt(3) and th.max() <= math.sqrt(3)
    # uniform: chi-square over 20 bins
    hist, _ = np.histogram(th, bins=20, range=(-math.sqrt(3), math.sqrt(3)))
    chi2 = ((hist - n / 20) ** 2 / (n / 20)).sum()
    assert chi2 < 45.0          # 19 dof, p ~ 1e-3
    for i, j in ((3, 9), (100, 2), (0, 77)):
        assert orc.theta(5, 11, i, j) == orc.theta(5, 11, j, i)
    assert orc.theta(5, 11, 3, 9) != orc.theta(5, 12, 3, 9)
    assert orc.theta(5, 11, 3, 9) != orc.theta(6, 11, 3, 9)


def test_philox_known_answers(orc):
    """Philox4x32-10 reproduces the known-answer vectors published with its
    definition (tests/golden/philox4x32_10_kat.txt): a wrong multiplier, key
    bump, word swap or round count changes every output word."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        assert orc.philox4x32_10(w[0:4], w[4:6]) == w[6:10], r


def test_philox_avalanche(orc):
    """Philox4x32-10 is a keyed bijection with full diffusion after 10 rounds:
    flipping one counter or key bit flips about half of the 128 output bits."""
    rng = np.random.default_rng(1)
    flips = []
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2)]
        base = orc.philox4x32_10(ctr, key)
        w, b = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        c2, k2 = list(ctr), list(key)
        if w < 4:
            c2[w] ^= 1 << b
        else:
            k2[w - 4] ^= 1 << b
        out = orc.philox4x32_10(c2, k2)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(base, out)))
    assert abs(np.mean(flips) - 64.0) < 2.0
    # distinct counters give distinct outputs (bijection on the counter)
    outs = {tuple(orc.philox4x32_10([i, 0, 0, 0], [9, 9])) for i in range(2000)}
    assert len(outs) == 2000


def test_pair_forces_obey_newton_third_law(orc):
    pos, vel, types, L = _box()
    D = orc.DpdParams(a=np.array([[25.0]]), gamma=4.5, sigma=3.0, dt=0.04, seed=9)
    F, E2 = orc.dpd_forces(_P(orc, L), D, pos, vel, types, step=3)
    assert np.abs(F.sum(0)).max() < 1e-11 * np.abs(F).max() * len(F)
    assert E2[0] > 0


def test_conservative_force_is_minus_gradient(orc):
    """Eq. 3 with w^C = 1 - r: F^C = -grad of sum a_ij (1-r)^2/2."""
    pos, vel, types, L = _box(n=60, L=4.0, seed=2)
    D = orc.DpdParams(a=np.array([[25.0]]), gamma=0.0, sigma=0.0, dt=0.04)
    P = _P(orc, L)
    F0, _ = orc.dpd_forces(P, D, pos, vel, types)
    h = 1e-6
    for i in range(4):
        for t in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, t] += h
            xm[i, t] -= h
            ep = orc.dpd_forces(P, D, xp, vel, types)[1][0]
            em = orc.dpd_forces(P, D, xm, vel, types)[1][0]
            assert abs(-(ep - em) / (2 * h) - F0[i, t]) < 1e-6 * max(1.0, abs(F0[i, t]))


def test_bond_force_is_minus_gradient(orc):
    pos, vel, types, L = _box(n=10, L=4.0, seed=3)
    bonds = np.array([[0, 1], [1, 2], [5, 9]])
    D = orc.DpdParams(a=np.array([[0.0]]), gamma=0.0, sigma=0.0, dt=0.04, K_bond=4.0, r0_bond=0.7)
    P = _P(orc, L)
    F0, E0 = orc.dpd_forces(P, D, pos, vel, types, bonds)
    h = 1e-6
    for i in (0, 1, 2, 5, 9, 4):
        for t in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, t] += h
            xm[i, t] -= h
            ep = orc.dpd_forces(P, D, xp, vel, types, bonds)[1][1]
            em = orc.dpd_forces(P, D, xm, vel, types, bonds)[1][1]
            assert abs(-(ep - em) / (2 * h) - F0[i, t]) < 1e-6 * max(1.0, abs(F0[i, t]))


def test_dissipative_force_direction(orc):
    """Eq. 4: two approaching beads are pushed apart by F^D, proportionally to
    gamma (1-r)^2 (v_ij . r_hat)."""
    L = 5.0
    pos = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]])
    vel = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    D = orc.DpdParams(a=np.array([[0.0]]), gamma=4.5, sigma=0.0, dt=0.04)
    F, _ = orc.dpd_forces(_P(orc, L), D, pos, vel, np.zeros(2, dtype=np.int32))
    # v_ij . r_hat = (2)(-1) = -2 ; F_i^D = -gamma w^2 (-2) r_hat_ij, r_hat_ij = -x
    assert abs(F[0, 0] - (-4.5 * 0.25 * 2.0)) < 1e-14
    assert abs(F[1, 0] + F[0, 0]) < 1e-14


def test_integrator_free_flight_and_oscillator(orc):
    """Table 2 with zero forces is free flight; with one harmonic bond and no
    DPD forces the scheme is velocity Verlet, which keeps the energy bounded
    (O(dt^2)) and the period of a spring of reduced mass 1/2."""
    L = 20.0
    P = orc.EwaldParams(L=L, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=2)
    types = np.zeros(2, dtype=np.int32)
    q = np.zeros(2)
    pos = np.array([[5.0, 5.0, 5.0], [6.0, 5.0, 5.0]])
    vel = np.array([[0.3, -0.2, 0.1], [0.1, 0.2, -0.4]])
    D0 = orc.DpdParams(a=np.array([[0.0]]), gamma=0.0, sigma=0.0, dt=0.01)
    F = np.zeros((2, 3))
    p1, v1, _, st, _ = orc.dpd_run(P, D0, pos, vel, F, types, q, nsteps=50)
    assert np.allclose(p1, pos + 50 * 0.01 * vel, atol=1e-12) and np.array_equal(v1, vel)
    assert st == 50
    # harmonic spring, r0 = 0, K = 4: omega = sqrt(2K) (reduced mass 1/2)
    K = 4.0
    D = orc.DpdParams(a=np.array([[0.0]]), gamma=0.0, sigma=0.0, dt=0.001, K_bond=K, r0_bond=0.0)
    bonds = np.array([[0, 1]])
    vel = np.zeros((2, 3))
    F, _ = orc.total_forces(P, D, pos, vel, types, q, bonds)
    nsteps = int(round(2 * math.pi / math.sqrt(2 * K) / 0.001))
    p1, v1, F1, _, _ = orc.dpd_run(P, D, pos, vel, F, types, q, bonds, nsteps=nsteps)
    assert np.abs(p1 - pos).max() < 2e-3          # back after one period
    e = lambda p, v: 0.5 * (v ** 2).sum() + 0.5 * K * ((p[0] - p[1]) ** 2).sum()
    assert abs(e(p1, v1) - e(pos, vel)) < 1e-5 * e(pos, vel)


def test_restart_equals_continuous_run(orc):
    """Counter-based noise: 2 + 2 steps reproduce 4 steps exactly."""
    s = W.polyelectrolyte(L=6.0, n_chains=2, chain_len=10, f=0.5, salt_fraction=0.05)
    P = orc.EwaldParams(L=s.L, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=s.M, p=2)
    dp = W.dpd_params(5)
    D = orc.DpdParams(**{k: v for k, v in dp.items()})
    F, _ = orc.total_forces(P, D, s.pos, s.vel, s.types, s.q, s.bonds)
    a = orc.dpd_run(P, D, s.pos, s.vel, F, s.types, s.q, s.bonds, step=0, nsteps=4)
    b = orc.dpd_run(P, D, s.pos, s.vel, F, s.types, s.q, s.bonds, step=0, nsteps=2)
    b = orc.dpd_run(P, D, b[0], b[1], b[2], s.types, s.q, s.bonds, step=b[3], nsteps=2)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3] == b[3] == 4


@pytest.mark.slow
def test_thermostat_temperature(orc):
    """Eq. 6 (sigma^2 = 2 gamma kT) with the Table 2 integrator keeps kT near 1
    at dt = 0.04 (Groot-Warren parameters), within a few percent."""
    n, L = 375, 5.0
    rng = np.random.default_rng(8)
    pos = rng.uniform(0, L, (n, 3))
    vel = rng.normal(0, 1, (n, 3))
    vel -= vel.mean(0)
    types = np.zeros(n, dtype=np.int32)
    q = np.zeros(n)
    P = orc.EwaldParams(L=L, alpha=1.0, r_cut=2.5, beta=4.0, kappa=1.0, M=16, p=2)
    D = orc.DpdParams(a=np.array([[25.0]]), gamma=4.5, sigma=3.0, dt=0.04, seed=17)
    F, _ = orc.total_forces(P, D, pos, vel, types, q)
    st = 0
    temps = []
    for blk in range(30):
        pos, vel, F, st, _ = orc.dpd_run(P, D, pos, vel, F, types, q, step=st, nsteps=10)
        if blk >= 10:
            temps.append((vel ** 2).sum() / (3 * n))
    assert abs(np.mean(temps) - 1.0) < 0.05
