"""Pin of the oracle's virial (reading c15; the paper is silent on it).

The virial the oracle reports is W = -L dE/dL with the beads' fractional
coordinates held fixed. Every part of it (real-space pairs, the direct and the
ENUF reciprocal sums, the k-space Slater form, the neutralising background) is
checked here against a central difference of the oracle's own energy in L,
which is pinned elsewhere (Madelung, alpha-independence, F = -grad E). The
difference quotient knows nothing of the closed forms it checks: a dropped
term, a wrong sign or a wrong power of L in any of them fails.
"""
import dataclasses

import numpy as np
import pytest

H = 1e-5   # relative step in L: truncation ~H^2, rounding ~1e-16/H of the energy


def _system(seed, n, L, net=0.0):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.0, 1.0, (n, 3))            # fractional coordinates
    q = np.array([1.0, -1.0] * (n // 2))
    q[0] += net
    return s, q


def _far_from_cutoff(s, L, rc, h=H):
    """No pair distance moves across r_c when L changes by a factor 1 +- h."""
    d = s[:, None, :] - s[None, :, :]
    d -= np.round(d)
    r = L * np.sqrt((d ** 2).sum(-1))
    r = r[np.triu_indices(len(s), 1)]
    return np.abs(r - rc).min() > 20 * h * rc


def _parts(orc, P, s, q):
    """(E, W) of each part at box edge P.L, positions s * L."""
    pos = s * P.L
    _, ER = orc.real_space(P, pos, q)
    _, EKd = orc.recip_direct(P, pos, q)
    _, EKe, _, _ = orc.recip_enuf(P, pos, q)
    ES = orc.self_neutral(P, q)
    return {"real": (ER[0], ER[1]), "recip_direct": (EKd[0], EKd[1]), "recip_enuf": (EKe[0], EKe[1]),
            "neutral": (ES[1], ES[2]), "self": (ES[0], 0.0)}


CASES = {
    # point charges, neutral
    "point_neutral": dict(alpha=1.8, r_cut=3.0, beta=0.0, kappa=1.0, M=16, p=4, net=0.0),
    # Slater correction in real space (beta = 4), net charge: background term
    "slater_real_net": dict(alpha=1.8, r_cut=3.0, beta=4.0, kappa=1.1, M=16, p=4, net=1.0),
    # the paper's beta = 1.125 and alpha, whose real-space pair term is still
    # 1e-3 at the cutoff: the system is chosen with no pair near r_c
    "paper_beta": dict(alpha=1.566, r_cut=3.0, beta=1.125, kappa=1.0 / (4 * np.pi), M=16, p=2, net=0.0),
    # Slater form factor in k space, net charge, spherical mode set
    "slater_k_net": dict(alpha=1.8, r_cut=3.0, beta=4.0, kappa=1.1, M=16, p=4, net=-1.0, slater_k=1, kmask=1),
    "slater_k_paper_beta": dict(alpha=1.566, r_cut=3.0, beta=1.125, kappa=1.0, M=12, p=3, net=1.0, slater_k=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_virial_is_minus_L_dE_dL(orc, name):
    spec = dict(CASES[name])
    net = spec.pop("net")
    L = 10.0
    n = 24 if spec.get("slater_k") else 40
    seed = 0
    s, q = _system(100 + seed, n, L, net)
    while not _far_from_cutoff(s, L, spec["r_cut"]):
        seed += 1
        s, q = _system(100 + seed, n, L, net)
    P = orc.EwaldParams(L=L, **spec)
    mid = _parts(orc, P, s, q)
    up = _parts(orc, dataclasses.replace(P, L=L * (1 + H)), s, q)
    dn = _parts(orc, dataclasses.replace(P, L=L * (1 - H)), s, q)
    tot_fd = tot_w = scale = 0.0
    for part in ("real", "recip_direct", "recip_enuf", "neutral", "self"):
        E, Wv = mid[part]
        w_fd = -(up[part][0] - dn[part][0]) / (2 * H)       # -L dE/dL
        tol = 1e-7 * (abs(E) + abs(Wv)) + 1e-13
        assert abs(Wv - w_fd) < tol, (part, Wv, w_fd)
        if part != "recip_direct":
            tot_fd += w_fd
            tot_w += Wv
            scale += abs(E) + abs(Wv)
    # the total the library reports: W_real + W_recip + W_neutral
    _, _, W_tot = orc.electrostatics(P, s * L, q, recip="enuf")
    assert abs(W_tot - tot_w) < 1e-12 * scale
    assert abs(W_tot - tot_fd) < 1e-7 * scale
    if net != 0.0:
        assert abs(mid["neutral"][0]) > 0.0


def test_virial_of_a_pair_is_r_times_force(orc):
    """Two charges alone in a large box, point charges, alpha small enough
    that the real-space term is the whole Coulomb pair inside r_c: W = r f(r)
    with f the Coulomb force magnitude kappa q_i q_j / r^2, i.e. W = E."""
    L = 40.0
    P = orc.EwaldParams(L=L, alpha=1e-4, r_cut=10.0, beta=0.0, kappa=1.3, M=4, p=2)
    pos = np.array([[1.0, 1.0, 1.0], [3.5, 1.0, 1.0]])
    q = np.array([1.0, -2.0])
    _, ER = orc.real_space(P, pos, q)
    E_coul = 1.3 * (1.0 * -2.0) / 2.5
    assert abs(ER[0] - E_coul) < 1e-3 * abs(E_coul)
    assert abs(ER[1] - ER[0]) < 1e-3 * abs(E_coul)
