"""Pins of the oracle's direct Ewald sum and Slater kernel (CPU only).

Each test checks the oracle against something other than itself: a literature
constant, a closed form, an exact invariance, or a finite-difference gradient.
"""
import math
import os

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    with open(os.path.join(GOLD, "madelung_nacl.txt")) as fh:
        return float([l for l in fh if not l.startswith("#")][0])


@pytest.mark.parametrize("k,M", [(2, 48), (3, 72)])
def test_madelung_rock_salt(orc, k, M):
    """Sec. 5: the Ewald energy of a rock-salt lattice of point charges gives
    the Madelung constant (golden value, literature)."""
    pos, q, L = W.rock_salt(k)
    P = orc.EwaldParams(L=L, alpha=3.0, r_cut=L / 2, beta=0.0, kappa=1.0, M=M, p=4)
    F, E, _ = orc.electrostatics(P, pos, q, recip="direct")
    m = -2.0 * E[3] / len(q)
    assert abs(m - _madelung()) / _madelung() < 1e-10
    # every ion sits at a centre of inversion: zero force
    assert np.abs(F).max() < 1e-12


def test_alpha_independence(orc):
    """Eq. 16: the total energy does not depend on the splitting parameter."""
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 10.0, (40, 3))
    q = np.array([1.0, -1.0] * 20)
    Es = []
    for a in (1.0, 1.3):
        P = orc.EwaldParams(L=10.0, alpha=a, r_cut=5.0, beta=1.125, kappa=1.0, M=56, p=4)
        Es.append(orc.electrostatics(P, pos, q, recip="direct")[1][3])
    assert abs(Es[0] - Es[1]) / abs(Es[0]) < 1e-11


def _small_system(seed=5, n=20, L=6.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, (n, 3)), np.array([1.0, -1.0] * (n // 2)), L


def test_forces_are_minus_gradient(orc):
    """Eq. 22 and the corrected Eq. 32: F = -grad E (central differences)."""
    pos, q, L = _small_system()
    P = orc.EwaldParams(L=L, alpha=1.2, r_cut=3.0, beta=4.0, kappa=1.1, M=16, p=4)
    # no pair within 1e-3 of the cutoff, so E is smooth along every probe
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    assert np.abs(r - 3.0).min() > 1e-3
    E0, F0 = None, None
    F0 = orc.electrostatics(P, pos, q, recip="direct")[0]
    h = 1e-5
    scale = np.abs(F0).max()
    for i in range(6):
        for t in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, t] += h
            xm[i, t] -= h
            ep = orc.electrostatics(P, xp, q, recip="direct")[1][3]
            em = orc.electrostatics(P, xm, q, recip="direct")[1][3]
            assert abs(-(ep - em) / (2 * h) - F0[i, t]) / scale < 1e-7


def test_net_force_and_translation_invariance(orc):
    pos, q, L = _small_system(seed=7)
    P = orc.EwaldParams(L=L, alpha=1.2, r_cut=3.0, beta=1.125, kappa=1.0, M=16, p=4)
    F0, E0, _ = orc.electrostatics(P, pos, q, recip="direct")
    assert np.abs(F0.sum(0)).max() < 1e-12 * max(1.0, np.abs(F0).max())
    shift = np.array([1.37, -2.21, 0.93])
    F1, E1, _ = orc.electrostatics(P, pos + shift, q, recip="direct")
    assert abs(E1[3] - E0[3]) < 1e-12 * abs(E0[3])
    assert np.abs(F1 - F0).max() < 1e-12 * np.abs(F0).max()


@pytest.mark.parametrize("r", [1e-3, 0.25, 0.5, 1.0, 2.0])
def test_two_smeared_charges_in_a_large_box(orc, r):
    """Eq. 27/28 through the whole periodic sum: a +1/-1 pair in a box of edge
    60 has the isolated Slater pair energy and force, shifted by the tin-foil
    dipole term -2 pi r^2 / (3V) (force 4 pi r/(3V)), up to O(r^4/L^5)."""
    L, beta = 60.0, 1.125
    P = orc.EwaldParams(L=L, alpha=0.3, r_cut=20.0, beta=beta, kappa=1.0, M=76, p=4)
    pos = np.array([[30.0, 30.0, 30.0], [30.0 + r, 30.0, 30.0]])
    q = np.array([1.0, -1.0])
    F, E, _ = orc.electrostatics(P, pos, q, recip="direct")
    V = L ** 3
    e_iso = -orc.slater_energy(beta, r)
    f_iso = orc.slater_force(beta, r)          # attraction: +x on the +1 charge
    tol = 1e-8 * (1.0 + r ** 4)                  # next term of the expansion ~ r^4/L^5
    assert abs(E[3] - (e_iso - 2 * math.pi * r * r / (3 * V))) < tol
    assert abs(F[0, 0] - (f_iso - 4 * math.pi * r / (3 * V))) < tol
    assert abs(F[0, 1]) < 1e-12 and abs(F[0, 2]) < 1e-12


def test_slater_limits_and_cutoff(orc):
    """Sec. 4: U(0) = kappa q_i q_j beta, F(0) = 0; B1, B2 -> 1 at large r (Fig. 2).
    Near r = 0, B2 = (2 beta r)^3/6 + O(r^4), so F(r)/r -> 4 beta^3/3."""
    for beta in (1.125, 4.0):
        assert abs(orc.slater_energy(beta, 1e-7) - beta) < 1e-6
        r = 1e-4
        assert abs(orc.slater_force(beta, r) / r - 4.0 * beta ** 3 / 3.0) < 1e-2 * beta ** 3
        b1 = [orc.B1(beta, r) for r in np.linspace(0.01, 6, 200)]
        b2 = [orc.B2(beta, r) for r in np.linspace(0.01, 6, 200)]
        assert np.all(np.diff(b1) >= 0) and np.all(np.diff(b2) >= 0)
        assert 0.99 < orc.B1(beta, 3.0) <= 1.0 and 0.96 < orc.B2(beta, 3.0) <= 1.0
    assert orc.B1(0.0, 0.3) == 1.0 and orc.B2(0.0, 0.3) == 1.0


def test_slater_potential_solves_poisson(orc):
    """Eq. 26 -> Eq. 27: phi(r) = B1/r solves the radial Poisson equation
    (1/r^2) d/dr (r^2 dphi/dr) = -4 pi rho with rho = beta^3/pi e^{-2 beta r}
    (unit charge, 4 pi eps0 eps_r = 1), checked by finite differences; and
    B2 = B1 - r dB1/dr, i.e. Eq. 28 is -d/dr of Eq. 27."""
    beta = 1.125
    h = 1e-3
    for r in (0.3, 0.8, 1.5, 2.5):
        phi = lambda s: orc.slater_energy(beta, s)
        flux = lambda s: s * s * (phi(s + h) - phi(s - h)) / (2 * h)
        lap = (flux(r + h) - flux(r - h)) / (2 * h) / (r * r)
        rho = beta ** 3 / math.pi * math.exp(-2 * beta * r)
        assert abs(lap + 4 * math.pi * rho) < 1e-5 * max(1.0, 4 * math.pi * rho)
        dB1 = (orc.B1(beta, r + 1e-6) - orc.B1(beta, r - 1e-6)) / 2e-6
        assert abs(orc.B2(beta, r) - (orc.B1(beta, r) - r * dB1)) < 1e-8


def test_self_and_neutral_terms(orc):
    """Eq. 16 third term; the background term vanishes for a neutral system and
    makes a net-charged total alpha-independent."""
    P = orc.EwaldParams(L=8.0, alpha=1.0, r_cut=4.0, beta=0.0, kappa=1.0, M=48, p=4)
    q = np.array([1.0, -1.0, 2.0, -2.0])
    out = orc.self_neutral(P, q)
    assert abs(out[0] + 10.0 / math.sqrt(math.pi)) < 1e-14 and out[1] == 0.0
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 8.0, (5, 3))
    qn = np.array([1.0, -1.0, 1.0, 1.0, -0.5])        # net charge 1.5
    Es = []
    for a in (1.2, 1.5):
        P.alpha = a
        Es.append(orc.electrostatics(P, pos, qn, recip="direct")[1][3])
    assert abs(Es[0] - Es[1]) < 1e-10
