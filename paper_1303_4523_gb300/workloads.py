"""Seeded synthetic inputs for the ENUF-DPD hot path.

This module holds no arithmetic of the method: it only draws positions,
velocities, charges, bead types and chain topologies with numpy's PCG64 and
returns plain arrays plus parameter sets. Both the CUDA path's tests/bench and
the oracle's tests take their inputs from here, so the two sides see the same
numbers.

Workload shapes follow the paper's simulated systems (Table 3: DPD boxes at
number density 3-4, a fraction of the beads carrying +-1 or multivalent
charges, polyelectrolyte chains with harmonic bonds).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1303

# Table 1 / Sec. 5 parameter sets, in reduced units (R_c = 1).
#   "paper":    alpha = 0.20 A^-1 * 7.829 A = 1.566, r_c = 3, p = 2, n_c = 7 (M = 16),
#               beta = 1.125 (lambda_e = 6.954 A), eps0 eps_r = 1 -> kappa = 1/(4 pi).
#   "bench":    alpha = 0.975, r_c = 3, p = 4, lambda = 0.25 (beta = 4),
#               kappa = Gamma/(4 pi) with Gamma = 13.87, M from the grid rule.
PAPER_SET = dict(alpha=1.566, r_cut=3.0, p=2, beta=1.125, kappa=1.0 / (4.0 * math.pi))
BENCH_SET = dict(alpha=0.975, r_cut=3.0, p=4, beta=4.0, kappa=13.87 / (4.0 * math.pi))

# DPD parameters of the polyelectrolyte run (Groot-Warren values).
DPD_SET = dict(a=25.0, gamma=4.5, sigma=3.0, dt=0.04, lambda_vv=0.65, K_bond=4.0, r0_bond=0.0)


def _smooth(m: int) -> bool:
    for f in (2, 3, 5):
        while m % f == 0:
            m //= f
    return m == 1


def grid_rule(L: float) -> int:
    """Base grid M = 1.6 L rounded to the nearest even 2^a 3^b 5^c integer
    (about one grid point per 0.6 R_c; 16 at L = 10, i.e. n_c = 7)."""
    target = 1.6 * L
    best = None
    for m in range(2, int(4 * target) + 8, 2):
        if not _smooth(m):
            continue
        if best is None or abs(m - target) < abs(best - target) - 1e-12:
            best = m
    return max(best, 8)


@dataclass
class System:
    """One synthetic DPD system. Arrays are float64 numpy; cast as needed."""
    name: str
    L: float
    pos: np.ndarray            # (N, 3)
    vel: np.ndarray            # (N, 3)
    q: np.ndarray              # (N,)
    types: np.ndarray          # (N,) int32
    bonds: np.ndarray          # (nb, 2) int32
    M: int
    params: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.q.shape[0])

    @property
    def n_charged(self) -> int:
        return int(np.count_nonzero(self.q))


def _rng(seed_offset: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))


def _velocities(rng, N, kT=1.0):
    v = rng.normal(0.0, math.sqrt(kT), size=(N, 3))
    return v - v.mean(axis=0, keepdims=True)


def electrolyte(N: int, L: float | None = None, n_charged: int | None = None,
                charged_fraction: float = 0.1, seed_offset: int = 1,
                pset: dict | None = None, M: int | None = None, valency: int = 1) -> System:
    """Uniform DPD beads in a periodic cube; a seeded subset carries charges.

    valency z: the charged subset is split into cations +z and anions -1 in the
    ratio 1 : z so that the system is neutral (z = 1 gives a +-1 electrolyte)."""
    rng = _rng(seed_offset)
    if L is None:
        L = (N / 3.0) ** (1.0 / 3.0)
    if n_charged is None:
        n_charged = int(round(charged_fraction * N))
    pos = rng.uniform(0.0, L, size=(N, 3))
    order = rng.permutation(N)
    q = np.zeros(N)
    n_cat = n_charged // (1 + valency)
    n_an = valency * n_cat
    q[order[:n_cat]] = float(valency)
    q[order[n_cat:n_cat + n_an]] = -1.0
    types = np.zeros(N, dtype=np.int32)
    types[q != 0] = 1
    return System(name=f"electrolyte N={N} L={L:.4g}", L=float(L), pos=pos,
                  vel=_velocities(rng, N), q=q, types=types,
                  bonds=np.zeros((0, 2), dtype=np.int32),
                  M=M if M is not None else grid_rule(L), params=dict(pset or BENCH_SET))


def electrolyte_small(pset: str = "bench") -> System:
    """N = 3000 beads, L = 10, 300 charged (150 +1, 150 -1): density 3."""
    ps = PAPER_SET if pset == "paper" else BENCH_SET
    return electrolyte(3000, 10.0, n_charged=300, seed_offset=0, pset=ps, M=16)


def electrolyte_sweep(N: int) -> System:
    """Electrolyte scaling sweep at density 3, 10% charged +-1 (N = 3000 ... 375000)."""
    return electrolyte(N, seed_offset=1, charged_fraction=0.1)


def polyelectrolyte(L: float = 30.0, density: float = 3.0, n_chains: int = 10,
                    chain_len: int = 50, f: float = 0.5, salt_fraction: float = 0.1,
                    valency: int = 1, seed_offset: int = 2, step: float = 0.5) -> System:
    """Linear chains (harmonic bonds, random-walk start), charge fraction f
    (q = -1 on charged monomers, evenly spaced), +1 counterions, z:1 salt at
    salt_fraction of the beads, the rest neutral solvent.

    bead types: 0 solvent, 1 monomer, 2 counterion, 3 salt cation, 4 salt anion."""
    rng = _rng(seed_offset)
    N = int(round(density * L ** 3))
    pos = np.empty((N, 3))
    q = np.zeros(N)
    types = np.zeros(N, dtype=np.int32)
    bonds = []
    k = 0
    n_charged_mono = 0
    every = 0 if f <= 0 else max(1, int(round(1.0 / f)))
    for c in range(n_chains):
        start = rng.uniform(0.0, L, size=3)
        for m in range(chain_len):
            if m == 0:
                pos[k] = start
            else:
                d = rng.normal(size=3)
                pos[k] = pos[k - 1] + step * d / np.linalg.norm(d)
                bonds.append((k - 1, k))
            types[k] = 1
            if every and (m % every == 0) and n_charged_mono < int(round(f * n_chains * chain_len)):
                q[k] = -1.0
                n_charged_mono += 1
            k += 1
    # counterions
    for _ in range(n_charged_mono):
        pos[k] = rng.uniform(0.0, L, size=3)
        q[k] = 1.0
        types[k] = 2
        k += 1
    # z:1 salt at salt_fraction of the beads: cations +z, anions -1, neutral
    n_salt = int(round(salt_fraction * N))
    n_cat = n_salt // (1 + valency)
    n_an = valency * n_cat
    for _ in range(n_cat):
        pos[k] = rng.uniform(0.0, L, size=3)
        q[k] = float(valency)
        types[k] = 3
        k += 1
    for _ in range(n_an):
        pos[k] = rng.uniform(0.0, L, size=3)
        q[k] = -1.0
        types[k] = 4
        k += 1
    # solvent
    ns = N - k
    pos[k:] = rng.uniform(0.0, L, size=(ns, 3))
    pos = np.mod(pos, L)
    return System(name=f"polyelectrolyte N={N} L={L:g} chains={n_chains}x{chain_len} f={f}",
                  L=float(L), pos=pos, vel=_velocities(rng, N), q=q, types=types,
                  bonds=np.asarray(bonds, dtype=np.int32).reshape(-1, 2),
                  M=grid_rule(L), params=dict(BENCH_SET))


def batch_sweep(n_systems: int = 64, n_min: int = 3000, n_max: int = 81000,
                seed_offset: int = 3) -> list[System]:
    """Uneven systems with N log-uniform in [n_min, n_max], each with its own box
    and grid. Even-indexed: z:1 electrolytes (about 10% of beads charged);
    odd-indexed: polyelectrolytes (chains of 50 beads, ~0.6% of beads) with
    charge fraction f in {0.25, 0.5, 1.0} and z:1 salt at 0.1 bead fraction.
    z in {1, 2} and f are drawn from the seed."""
    rng = _rng(seed_offset)
    out = []
    for s in range(n_systems):
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = (N / 3.0) ** (1.0 / 3.0)
        z = int(rng.choice([1, 2]))
        if s % 2 == 0:
            sysm = electrolyte(N, L, charged_fraction=0.1, seed_offset=100 + s, valency=z)
        else:
            fch = float(rng.choice([0.25, 0.5, 1.0]))
            n_chains = max(1, int(round(0.006 * N / 50)))
            sysm = polyelectrolyte(L=L, n_chains=n_chains, f=fch, salt_fraction=0.1,
                                   valency=z, seed_offset=100 + s)
        sysm.name = f"batch[{s}] " + sysm.name
        out.append(sysm)
    return out


def rock_salt(k: int, d: float = 1.0):
    """Rock-salt lattice: (2k)^3 sites of a simple cubic lattice with spacing d,
    charges alternating +-1 (two interpenetrating FCC sublattices).
    Returns (pos, q, L)."""
    m = 2 * k
    idx = np.array([(i, j, l) for i in range(m) for j in range(m) for l in range(m)], dtype=np.float64)
    q = np.where(idx.sum(axis=1).astype(int) % 2 == 0, 1.0, -1.0)
    return idx * d, q, m * d


def dpd_params(ntypes: int, seed: int = 1303, **over) -> dict:
    """Conservative matrix a_ij = a for every type pair, plus the DPD set."""
    ps = dict(DPD_SET)
    ps.update(over)
    a = np.full((ntypes, ntypes), ps.pop("a"))
    ps["a"] = a
    ps["seed"] = seed
    return ps


# Table 1 DPD parameters of the paper's own runs (density 4, R_c = 7.829 A):
# a_ii = 78.67, a_ij = a_ii + 2.05 chi with chi = 0.87 between the
# polyelectrolyte and the solvent, gamma = 6.74, sigma = 3.67, dt = 0.02,
# lambda = 0.65, harmonic bonds K^S = 64 about r_eq = 0.7 (Sec. 5).
PAPER_DPD = dict(a_ii=78.67, chi=0.87, gamma=6.74, sigma=3.67, dt=0.02, lambda_vv=0.65,
                 K_bond=64.0, r0_bond=0.7)


def paper_dpd_params(seed: int = 1303) -> dict:
    """DPD parameters of Table 1 for bead types 0 solvent, 1 monomer, 2
    counterion, 3 salt cation, 4 salt anion: every pair a_ii except monomer
    with any other type, a_ii + 2.05 chi."""
    p = PAPER_DPD
    a = np.full((5, 5), p["a_ii"])
    a_ps = p["a_ii"] + 2.05 * p["chi"]
    for t in (0, 2, 3, 4):
        a[1, t] = a[t, 1] = a_ps
    return dict(a=a, gamma=p["gamma"], sigma=p["sigma"], dt=p["dt"], lambda_vv=p["lambda_vv"],
                K_bond=p["K_bond"], r0_bond=p["r0_bond"], seed=seed)


def single_polyelectrolyte(f: float, L: float = 30.0, density: float = 4.0, n_p: int = 48,
                           seed_offset: int = 60, theta: float = 0.0, valency: int = 1) -> System:
    """Table 3 set 5 (Sec. 5): one chain of n_p beads (random walk with the bond
    length r_eq = 0.7), round(f n_p) of them evenly spaced with q = -1, as many
    +1 counterions, the rest neutral solvent (N = density L^3). Set 6: added
    Z:1 salt whose cations (+valency) carry theta times the chain's charge,
    round(theta f n_p / valency) of them, with theta f n_p anions (-1).
    Bead types: 0 solvent, 1 monomer, 2 counterion, 3 salt cation, 4 salt
    anion. Paper parameter set for the electrostatics, M from the grid rule."""
    rng = _rng(seed_offset)
    N = int(round(density * L ** 3))
    nq = int(round(f * n_p))
    pos = np.empty((N, 3))
    q = np.zeros(N)
    types = np.zeros(N, dtype=np.int32)
    start = rng.uniform(0.0, L, size=3)
    for m in range(n_p):
        if m == 0:
            pos[0] = start
        else:
            d = rng.normal(size=3)
            pos[m] = pos[m - 1] + PAPER_DPD["r0_bond"] * d / np.linalg.norm(d)
        types[m] = 1
    for k in range(nq):
        q[(k * n_p + n_p // 2) // nq if nq else 0] = -1.0
    pos[n_p:n_p + nq] = rng.uniform(0.0, L, size=(nq, 3))
    q[n_p:n_p + nq] = 1.0
    types[n_p:n_p + nq] = 2
    k = n_p + nq
    n_cat, n_an = int(round(theta * nq / valency)), int(round(theta * nq))
    q[k:k + n_cat], types[k:k + n_cat] = float(valency), 3
    q[k + n_cat:k + n_cat + n_an], types[k + n_cat:k + n_cat + n_an] = -1.0, 4
    pos[n_p + nq:] = rng.uniform(0.0, L, size=(N - n_p - nq, 3))
    pos = np.mod(pos, L)
    bonds = np.array([(m - 1, m) for m in range(1, n_p)], dtype=np.int32).reshape(-1, 2)
    return System(name=f"single polyelectrolyte N={N} L={L:g} N_p={n_p} f={f} salt theta={theta} z={valency}",
                  L=float(L), pos=pos, vel=_velocities(rng, N), q=q, types=types, bonds=bonds, M=grid_rule(L),
                  params=dict(PAPER_SET))


def electrolyte_rdf_system(L: float = 10.0, density: float = 4.0, n_ions: int = 132,
                           seed_offset: int = 61) -> System:
    """Table 3 set 3: N = density L^3 beads (4000 at L = 10), n_ions cations
    (+1, type 3), n_ions anions (-1, type 4), the rest neutral (type 0), all
    uniform; paper parameter set, M from the grid rule."""
    rng = _rng(seed_offset)
    N = int(round(density * L ** 3))
    pos = rng.uniform(0.0, L, size=(N, 3))
    q = np.zeros(N)
    types = np.zeros(N, dtype=np.int32)
    q[:n_ions], types[:n_ions] = 1.0, 3
    q[n_ions:2 * n_ions], types[n_ions:2 * n_ions] = -1.0, 4
    return System(name=f"electrolyte N={N} L={L:g} ions={n_ions}+{n_ions}", L=float(L), pos=pos,
                  vel=_velocities(rng, N), q=q, types=types, bonds=np.zeros((0, 2), np.int32),
                  M=grid_rule(L), params=dict(PAPER_SET))
