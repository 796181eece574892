"""Pins of the oracle's k-space Slater reading (CPU only).

Reading C moves the Slater smearing of Eq. 26-27 into k space: the influence
function gains the form factor rho(k) = (1 + k^2/(4 beta^2))^{-2} (the Fourier
transform of the Slater density whose potential is phi_S = B1/r, Eq. 27), and
the real-space kernel becomes phi_S(r) - I(r)/r with a radial quadrature I.
For untruncated sums it is an exact rewriting of the default reading (the
Slater correction in real space only), so the two must give the same total
energy, forces and virial; with rho = 1 the quadrature must reproduce erf.
"""
import math

import numpy as np
import pytest


def _system(n, L, seed, net=0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, (n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q[:net] = 1.0
    return pos, q


@pytest.mark.parametrize("alpha", [0.4, 0.975, 1.566])
def test_quadrature_reproduces_erf(orc, alpha):
    P = orc.EwaldParams(L=10.0, alpha=alpha, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=4, slater_k=1)
    for r in (0.05, 0.3, 1.0, 2.0, 3.0, 5.0):
        I, dI = orc.slater_I(P, r, rho_one=True)
        assert abs(I - math.erf(alpha * r)) < 1e-13
        assert abs(dI - 2 * alpha / math.sqrt(math.pi) * math.exp(-(alpha * r) ** 2)) < 1e-13
    _, d0 = orc.slater_I(P, 0.0, rho_one=True)
    assert abs(d0 - 2 * alpha / math.sqrt(math.pi)) < 1e-13


@pytest.mark.parametrize("beta,r_far,tol", [(1.125, 9.0, 1e-8), (4.0, 6.0, 1e-14)])
def test_far_field_is_the_slater_potential(orc, beta, r_far, tol):
    """Far out the k-space kernel I(r)/r is the potential of the smeared charge,
    phi_S(r) = (1 - (1 + beta r) e^{-2 beta r})/r (Eq. 27): the real-space kernel
    of Reading C, phi_S - I/r (a Slater-smeared erfc), decays monotonically to 0."""
    P = orc.EwaldParams(L=40.0, alpha=1.5, r_cut=12.0, beta=beta, kappa=1.0, M=16, p=4, slater_k=1)
    d = []
    for r in (1.0, 2.0, 3.0, 4.0, r_far):
        I, _ = orc.slater_I(P, r)
        d.append(abs(I / r - (1 - (1 + beta * r) * math.exp(-2 * beta * r)) / r))
    assert all(d[k + 1] < d[k] for k in range(3))
    assert d[-1] < tol


@pytest.mark.parametrize("case", [
    dict(L=10.0, alpha=1.2, r_cut=5.0, beta=4.0, M=48, n=120, net=0),
    dict(L=10.0, alpha=1.2, r_cut=5.0, beta=4.0, M=48, n=121, net=5),
    dict(L=30.0, alpha=0.4, r_cut=15.0, beta=1.125, M=48, n=80, net=0),
])
def test_reading_c_equals_reading_a(orc, case):
    c = dict(case)
    n, net = c.pop("n"), c.pop("net")
    pos, q = _system(n, c["L"], seed=n + net, net=net)
    PA = orc.EwaldParams(kappa=1.0, p=4, slater_k=0, **c)
    PC = orc.EwaldParams(kappa=1.0, p=4, slater_k=1, **c)
    FA, EA, WA = orc.electrostatics(PA, pos, q, recip="direct")
    FC, EC, WC = orc.electrostatics(PC, pos, q, recip="direct")
    # the pieces differ, the totals agree
    assert abs(EA[1] - EC[1]) > 1e-6 * abs(EA[3])
    assert abs(EC[3] - EA[3]) < 1e-10 * abs(EA[3])
    assert math.sqrt(((FC - FA) ** 2).sum() / (FA ** 2).sum()) < 1e-10
    assert abs(WC - WA) < 1e-9 * max(abs(WA), abs(EA[3]))


def test_enuf_with_form_factor_converges_to_direct(orc):
    pos, q = _system(300, 10.0, seed=7)
    P = orc.EwaldParams(L=10.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=8, slater_k=1)
    Fd, Ed = orc.recip_direct(P, pos, q)
    Fe, Ee, _, _ = orc.recip_enuf(P, pos, q)
    assert abs(Ee[0] - Ed[0]) < 1e-8 * abs(Ed[0])
    assert abs(Ee[1] - Ed[1]) < 1e-7 * abs(Ed[1])
    assert math.sqrt(((Fe - Fd) ** 2).sum() / (Fd ** 2).sum()) < 1e-8
