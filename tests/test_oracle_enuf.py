"""Pins of the oracle's naive ENUF (CPU only).

The NFFT approximation must converge to the direct Ewald sum as the window
cutoff p grows (the truncation error of a Gaussian window decays like
exp(-2 pi p / 3) at oversampling 2 -- Sec. 5: "the error decays exponentially
with p"); its DFT stages must agree with a library FFT applied to its own
spread grid; and its ik-differentiated forces must sum to zero.
"""
import math

import numpy as np
import pytest

from paper_1303_4523_gb300 import workloads as W


def _charged(s):
    ch = np.nonzero(s.q)[0]
    return s.pos[ch], s.q[ch]


@pytest.fixture(scope="module")
def small():
    s = W.electrolyte_small("bench")
    return s, *_charged(s)


def _params(orc, s, **kw):
    d = dict(L=s.L, M=s.M, **s.params)
    d.update(kw)
    return orc.EwaldParams(**d)


@pytest.mark.parametrize("M", [16, 32])
def test_enuf_converges_to_direct_ewald(orc, small, M):
    s, pos, q = small
    P = _params(orc, s, M=M)
    Fd, Ed = orc.recip_direct(P, pos, q)
    eE, eF = [], []
    for p in range(1, 9):
        P.p = p
        Fe, Ee, _, _ = orc.recip_enuf(P, pos, q)
        eE.append(abs(Ee[0] - Ed[0]) / abs(Ed[0]))
        eF.append(math.sqrt(((Fe - Fd) ** 2).sum() / (Fd ** 2).sum()))
    eE, eF = np.array(eE), np.array(eF)
    # monotone, at least a factor 5 per unit of p, and within the Gaussian
    # window's exp(-2 pi p/3) envelope (times a modest constant)
    assert np.all(eE[1:] < eE[:-1] / 5) and np.all(eF[1:] < eF[:-1] / 5)
    envelope = np.exp(-2 * math.pi * np.arange(1, 9) / 3)
    assert np.all(eF < 4.0 * envelope) and np.all(eE < 4.0 * envelope)
    assert eE[-1] < 1e-8 and eF[-1] < 1e-8


def test_enuf_virial_converges(orc, small):
    s, pos, q = small
    P = _params(orc, s, p=8)
    _, Ed = orc.recip_direct(P, pos, q)
    _, Ee, _, _ = orc.recip_enuf(P, pos, q)
    assert abs(Ee[1] - Ed[1]) / abs(Ed[1]) < 1e-7


def _lib_energy_and_field(P, grid):
    """Energy and conjugated field from the oracle's own grid, with numpy's FFT."""
    n = grid.shape[0]
    nc = P.M // 2 - 1
    b = 2.0 * P.sigma_s * P.p / ((2.0 * P.sigma_s - 1.0) * math.pi)
    Fh = np.fft.fftn(grid.transpose(2, 1, 0))          # axes (x, y, z), e^{-2 pi i k l/n}
    k = np.fft.fftfreq(n, 1.0 / n)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    mask = (np.abs(KX) <= nc) & (np.abs(KY) <= nc) & (np.abs(KZ) <= nc)
    mask &= (KX ** 2 + KY ** 2 + KZ ** 2) > 0
    K2 = np.where(mask, KX ** 2 + KY ** 2 + KZ ** 2, 1.0)
    c = np.exp(-b * (math.pi * KX / n) ** 2) * np.exp(-b * (math.pi * KY / n) ** 2) \
        * np.exp(-b * (math.pi * KZ / n) ** 2)
    f = np.where(mask, np.exp(-math.pi ** 2 * K2 / (P.alpha * P.L) ** 2) / K2, 0.0)
    S = Fh / c
    E = P.kappa / (2 * math.pi * P.L) * (f * np.abs(S) ** 2).sum()
    h = []
    for Ka in (KX, KY, KZ):
        G = Ka * f * S / c
        field = np.fft.ifftn(G) * n ** 3                 # e^{+2 pi i k l/n}, unnormalised
        h.append(field.imag.transpose(2, 1, 0))
    return E, np.array(h)


@pytest.mark.parametrize("M,p", [(8, 2), (16, 4)])
def test_enuf_dft_stages_match_library_fft(orc, small, M, p):
    s, pos, q = small
    P = _params(orc, s, M=M, p=p)
    F, EW, grid, h = orc.recip_enuf(P, pos, q, want_grid=True, want_h=True)
    E_lib, h_lib = _lib_energy_and_field(P, grid)
    assert abs(E_lib - EW[0]) / abs(EW[0]) < 1e-12
    assert np.abs(h - h_lib).max() < 1e-11 * np.abs(h_lib).max()


def test_enuf_spread_grid_total_charge(orc, small):
    """A single unit charge: the spread grid sums to (sum_a psi(frac + p - 1 - a))^3,
    which tends to 1 (the Gaussian window integrates to one) as p grows."""
    s, pos, q = small
    P = _params(orc, s)
    one = np.array([[1.234, 5.678, 9.012]])
    for p, tol in ((2, 1e-2), (4, 1e-4), (8, 1e-8)):
        P.p = p
        _, _, g1, _ = orc.recip_enuf(P, one, np.array([1.0]), want_grid=True)
        assert abs(g1.sum() - 1.0) < tol


def test_enuf_net_force_vanishes(orc, small):
    s, pos, q = small
    for p in (2, 4):
        P = _params(orc, s, p=p)
        F, _, _, _ = orc.recip_enuf(P, pos, q)
        assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).max() * len(q)


def test_enuf_madelung(orc):
    """Sec. 5 first simulation set, with the reciprocal part by ENUF."""
    with open("tests/golden/madelung_nacl.txt") as fh:
        m_ref = float([l for l in fh if not l.startswith("#")][0])
    pos, q, L = W.rock_salt(2)
    P = orc.EwaldParams(L=L, alpha=3.0, r_cut=L / 2, beta=0.0, kappa=1.0, M=48, p=8)
    F, E, _ = orc.electrostatics(P, pos, q, recip="enuf")
    assert abs(-2 * E[3] / len(q) - m_ref) / m_ref < 1e-7


def test_enuf_sampled_forces_match_full(orc, small):
    s, pos, q = small
    P = _params(orc, s)
    F, _, _, _ = orc.recip_enuf(P, pos, q)
    idx = np.array([0, 7, 123, 299])
    Fs, _, _, _ = orc.recip_enuf(P, pos, q, sample=idx)
    assert np.array_equal(F[idx], Fs)
    Fr, _ = orc.real_space(P, pos, q)
    Frs, _ = orc.real_space(P, pos, q, sample=idx)
    assert np.array_equal(Fr[idx], Frs)


def test_spherical_mask_converges(orc, small):
    s, pos, q = small
    P = _params(orc, s, kmask=1, p=8)
    Fd, Ed = orc.recip_direct(P, pos, q)
    Fe, Ee, _, _ = orc.recip_enuf(P, pos, q)
    assert abs(Ee[0] - Ed[0]) / abs(Ed[0]) < 1e-8
    P.kmask = 0
    _, Ec = orc.recip_direct(P, pos, q)
    assert Ed[0] != Ec[0]


# --- analytic-gradient forces (one inverse transform instead of three) -------


def _interior_beads(s, pos, P, k=4, margin=0.2):
    """Beads whose grid coordinate n x / L is at least `margin` from an integer
    in every dimension, so that a small move keeps the same 2p taps."""
    u = np.mod(pos, s.L) * P.ng / s.L
    fr = u - np.floor(u)
    ok = np.all((fr > margin) & (fr < 1 - margin), axis=1)
    return np.nonzero(ok)[0][:k]


@pytest.mark.parametrize("p", [2, 4, 6])
def test_gradient_mode_is_minus_gradient_of_the_nfft_energy(orc, small, p):
    """The gradient-mode force is the exact derivative of the oracle's own NFFT
    energy (which the convergence and Madelung tests pin): central differences
    of E_K in every coordinate of a few beads reproduce it."""
    s, pos, q = small
    P = _params(orc, s, p=p, deriv=1)
    F, EW, _, _ = orc.recip_enuf(P, pos, q)
    beads = _interior_beads(s, pos, P)
    assert len(beads) >= 3
    h = 1e-5
    fscale = np.abs(F).max()
    for i in beads:
        for a in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, a] += h
            xm[i, a] -= h
            Ep = orc.recip_enuf(P, xp, q)[1][0]
            Em = orc.recip_enuf(P, xm, q)[1][0]
            fd = -(Ep - Em) / (2 * h)
            assert abs(fd - F[i, a]) < 2e-7 * fscale, (p, i, a, fd, F[i, a])


@pytest.mark.parametrize("M", [16, 32])
def test_gradient_mode_converges_to_direct_ewald(orc, small, M):
    s, pos, q = small
    P = _params(orc, s, M=M, deriv=1)
    Fd, _ = orc.recip_direct(P, pos, q)
    eF = []
    for p in range(1, 9):
        P.p = p
        Fe, _, _, _ = orc.recip_enuf(P, pos, q)
        eF.append(math.sqrt(((Fe - Fd) ** 2).sum() / (Fd ** 2).sum()))
    eF = np.array(eF)
    # same exp(-2 pi p/3) envelope as the ik forces, with a larger constant: the
    # derivative of the window carries the factor 2 d / b (measured at M = 32:
    # eF / envelope = 14, 10, 7.0, 4.6, 3.2, 2.2, 1.5, 1.1 for p = 1..8)
    envelope = np.exp(-2 * math.pi * np.arange(1, 9) / 3)
    assert np.all(eF[1:] < eF[:-1] / 3)
    assert np.all(eF < 16.0 * envelope)
    assert eF[-1] < 1e-7


def test_gradient_mode_field_matches_library_fft(orc, small):
    """The one real field of the gradient mode, rebuilt from the oracle's own
    spread grid with numpy's FFT."""
    s, pos, q = small
    P = _params(orc, s, M=16, p=4, deriv=1)
    _, EW, grid, h = orc.recip_enuf(P, pos, q, want_grid=True, want_h=True)
    n = grid.shape[0]
    nc = P.M // 2 - 1
    b = 2.0 * P.sigma_s * P.p / ((2.0 * P.sigma_s - 1.0) * math.pi)
    Fh = np.fft.fftn(grid.transpose(2, 1, 0))
    k = np.fft.fftfreq(n, 1.0 / n)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    mask = (np.abs(KX) <= nc) & (np.abs(KY) <= nc) & (np.abs(KZ) <= nc) & (KX ** 2 + KY ** 2 + KZ ** 2 > 0)
    K2 = np.where(mask, KX ** 2 + KY ** 2 + KZ ** 2, 1.0)
    c = np.exp(-b * (math.pi / n) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    f = np.where(mask, np.exp(-math.pi ** 2 * K2 / (P.alpha * P.L) ** 2) / K2, 0.0)
    field = np.fft.ifftn(f * Fh / c ** 2) * n ** 3
    assert np.abs(field.imag).max() < 1e-10 * np.abs(field.real).max()
    assert np.abs(h[0] - field.real.transpose(2, 1, 0)).max() < 1e-11 * np.abs(field.real).max()


def test_gradient_and_ik_forces_agree_at_large_p(orc, small):
    s, pos, q = small
    Fi, Ei, _, _ = orc.recip_enuf(_params(orc, s, p=8), pos, q)
    Fg, Eg, _, _ = orc.recip_enuf(_params(orc, s, p=8, deriv=1), pos, q)
    assert Ei[0] == Eg[0] and Ei[1] == Eg[1]
    assert math.sqrt(((Fg - Fi) ** 2).sum() / (Fi ** 2).sum()) < 1e-7
