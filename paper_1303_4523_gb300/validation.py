"""Validation runs of Sec. 5 on the GPU path (structure of the simulated
systems, not parity): the mean radius of gyration of a single polyelectrolyte
against its charge fraction f (Table 3 set 5; the paper finds the fully
ionised chain ~1.31 times larger than the neutral one) and the radial
distribution functions of an electrolyte (Table 3 set 3; the paper observes
g_+-(r) g_++/--(r) = g_00(r)^2), and the chain's <Rg> under added Z:1 salt
(Table 3 set 6; the paper finds the chain contracting, most with trivalent
counterions, smallest near the neutralising ratio theta = 1).

The trajectories come from DpdSystem (the CUDA step); the analysis is plain
numpy on the host, on positions copied back every `every` steps.

    python -m paper_1303_4523_gb300.validation rg --f 0 1 --equil 50000 --steps 250000
    python -m paper_1303_4523_gb300.validation rg --f 1 --theta 0.5 1 --valency 3
    python -m paper_1303_4523_gb300.validation rdf --equil 10000 --steps 200000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as W


def radius_of_gyration(x: np.ndarray, L: float) -> float:
    """Radius of gyration of a chain given its bead positions in bond order
    (any periodic images): the chain is unwrapped by summing minimum-image bond
    vectors, then Rg^2 = mean |x - x_cm|^2."""
    x = np.asarray(x, np.float64)
    d = np.diff(x, axis=0)
    d -= L * np.rint(d / L)
    u = np.concatenate([x[:1], x[:1] + np.cumsum(d, axis=0)])
    c = u - u.mean(axis=0)
    return float(math.sqrt((c * c).sum(axis=1).mean()))


def pair_histogram(a: np.ndarray, b: np.ndarray | None, L: float, r_max: float, nbins: int) -> np.ndarray:
    """Counts of minimum-image distances in [0, r_max) in nbins equal bins:
    between all pairs i < j of a when b is None, else between a and b
    (r_max <= L/2)."""
    a = np.mod(np.asarray(a, np.float64), L)
    same = b is None
    b = a if same else np.mod(np.asarray(b, np.float64), L)
    edges = np.linspace(0.0, r_max, nbins + 1)
    try:
        from scipy.spatial import cKDTree
    except ImportError:
        cKDTree = None
    if cKDTree is not None:
        ta = cKDTree(a, boxsize=L)
        tb = ta if same else cKDTree(b, boxsize=L)
        dm = ta.sparse_distance_matrix(tb, r_max, output_type="ndarray")
        keep = dm["v"] < r_max
        if same:
            keep &= dm["i"] < dm["j"]
        h, _ = np.histogram(dm["v"][keep], bins=edges)
        return h.astype(np.float64)
    h = np.zeros(nbins)
    for i0 in range(0, a.shape[0], 512):
        d = a[i0:i0 + 512, None, :] - b[None, :, :]
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(axis=2))
        if same:
            r = r[np.arange(r.shape[0])[:, None] + i0 < np.arange(r.shape[1])[None, :]]
        h += np.histogram(r[r < r_max], bins=edges)[0]
    return h


def rdf_normalise(h: np.ndarray, n_a: int, n_b: int | None, L: float, r_max: float, frames: int = 1):
    """g(r) from pair counts summed over frames: counts over the ideal-gas
    expectation (pairs x shell volume / V); n_b None: pairs within one set."""
    nbins = h.shape[0]
    edges = np.linspace(0.0, r_max, nbins + 1)
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    pairs = n_a * (n_a - 1) / 2.0 if n_b is None else float(n_a) * n_b
    r = 0.5 * (edges[1:] + edges[:-1])
    return r, h / (frames * pairs * shell / L ** 3)


def block_sem(x: np.ndarray, blocks: int = 10) -> float:
    """Standard error of the mean of a correlated series from the spread of
    the means of `blocks` consecutive blocks."""
    x = np.asarray(x, np.float64)
    n = (x.shape[0] // blocks) * blocks
    if n < blocks or blocks < 2:
        return float("nan")
    m = x[:n].reshape(blocks, -1).mean(axis=1)
    return float(m.std(ddof=1) / math.sqrt(blocks))


def _system(enuf, s, prec, kappa, seed):
    P = dict(L=s.L, M=s.M, **s.params)
    if kappa is not None:
        P["kappa"] = kappa
    plan = enuf.Plan(enuf.make_params(prec=prec, **P), s.N)
    dp = W.paper_dpd_params(seed)
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q,
                          s.bonds, lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"],
                          seed=dp["seed"])
    return plan, sysm, P


def run_polyelectrolyte(f: float, steps: int, equil: int, every: int = 100, prec: str = "fp32",
                        kappa: float | None = None, seed: int = 1303, n_p: int = 48, theta: float = 0.0,
                        valency: int = 1) -> dict:
    """Table 3 set 5: one chain of n_p beads with charge fraction f in N =
    108000 beads (L = 30, density 4), Table 1 DPD parameters, the paper's
    electrostatic set (kappa overrides its coupling); set 6: added Z:1 salt
    at charge ratio theta. equil steps, then `steps` steps sampled every
    `every`: <Rg> with its block standard error, the mean bond length and kT
    from the kinetic energy."""
    from . import enuf
    s = W.single_polyelectrolyte(f, n_p=n_p, theta=theta, valency=valency)
    plan, sysm, P = _system(enuf, s, prec, kappa, seed)
    sysm.step(equil)
    pos = np.empty((s.N, 3), plan.dtype_np)
    rg, kin, bond = [], [], []
    t0 = time.perf_counter()
    for _ in range(max(1, steps // every)):
        E = sysm.step(every, want_energy=True)
        sysm.get_state_into(pos=pos)
        x = pos[:n_p].astype(np.float64)
        rg.append(radius_of_gyration(x, s.L))
        d = np.diff(x, axis=0)
        d -= s.L * np.rint(d / s.L)
        bond.append(float(np.sqrt((d * d).sum(axis=1)).mean()))
        kin.append(E[6])
    wall = time.perf_counter() - t0
    done = max(1, steps // every) * every
    sysm.close()
    plan.close()
    return {"run": "rg", "f": f, "theta": theta, "valency": valency, "n_p": n_p, "N": s.N, "L": s.L,
            "prec": prec, "kappa": P["kappa"],
            "equil": equil, "steps": done, "every": every, "rg_mean": float(np.mean(rg)),
            "rg_sem": block_sem(np.array(rg)), "bond_mean": float(np.mean(bond)),
            "kT": float(2.0 * np.mean(kin) / (3.0 * s.N)), "ms_per_step": 1000.0 * wall / done}


def run_electrolyte_rdf(steps: int, equil: int, every: int = 200, prec: str = "fp32",
                        kappa: float | None = None, seed: int = 1303, r_max: float = 3.0,
                        nbins: int = 60) -> dict:
    """Table 3 set 3: 132 cations, 132 anions and 3736 neutral beads in L = 10
    (density 4); g_00, g of equal-sign ions (++ and -- pooled) and g_+- over
    the run, and the paper's relation g_+- g_equal / g_00^2 where g_00 > 0.5."""
    from . import enuf
    s = W.electrolyte_rdf_system()
    plan, sysm, P = _system(enuf, s, prec, kappa, seed)
    sysm.step(equil)
    pos = np.empty((s.N, 3), plan.dtype_np)
    sel = {"0": s.q == 0, "+": s.q > 0, "-": s.q < 0}
    n = {k: int(v.sum()) for k, v in sel.items()}
    h = {k: np.zeros(nbins) for k in ("00", "++", "--", "+-")}
    kin, frames = [], 0
    t0 = time.perf_counter()
    for _ in range(max(1, steps // every)):
        E = sysm.step(every, want_energy=True)
        sysm.get_state_into(pos=pos)
        x = pos.astype(np.float64)
        h["00"] += pair_histogram(x[sel["0"]], None, s.L, r_max, nbins)
        h["++"] += pair_histogram(x[sel["+"]], None, s.L, r_max, nbins)
        h["--"] += pair_histogram(x[sel["-"]], None, s.L, r_max, nbins)
        h["+-"] += pair_histogram(x[sel["+"]], x[sel["-"]], s.L, r_max, nbins)
        kin.append(E[6])
        frames += 1
    wall = time.perf_counter() - t0
    sysm.close()
    plan.close()
    r, g00 = rdf_normalise(h["00"], n["0"], None, s.L, r_max, frames)
    _, gpp = rdf_normalise(h["++"], n["+"], None, s.L, r_max, frames)
    _, gmm = rdf_normalise(h["--"], n["-"], None, s.L, r_max, frames)
    _, gpm = rdf_normalise(h["+-"], n["+"], n["-"], s.L, r_max, frames)
    geq = 0.5 * (gpp + gmm)
    ok = g00 > 0.5
    rel = gpm[ok] * geq[ok] / g00[ok] ** 2
    return {"run": "rdf", "N": s.N, "L": s.L, "prec": prec, "kappa": P["kappa"], "equil": equil,
            "steps": frames * every, "every": every, "r": r.round(4).tolist(), "g00": g00.round(4).tolist(),
            "g_equal": geq.round(4).tolist(), "g_opposite": gpm.round(4).tolist(),
            "relation_mean": float(rel.mean()), "relation_max_dev": float(np.abs(rel - 1.0).max()),
            "kT": float(2.0 * np.mean(kin) / (3.0 * s.N)), "ms_per_step": 1000.0 * wall / (frames * every)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("run", choices=["rg", "rdf"])
    ap.add_argument("--f", type=float, nargs="*", default=[0.0, 1.0], help="charge fractions (rg)")
    ap.add_argument("--theta", type=float, nargs="*", default=[0.0], help="added-salt charge ratios (rg)")
    ap.add_argument("--valency", type=int, default=1, help="salt cation valency (rg)")
    ap.add_argument("--steps", type=int, default=250000)
    ap.add_argument("--equil", type=int, default=50000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kappa", type=float, default=None, help="Coulomb coupling (default: the paper set's 1/4pi)")
    a = ap.parse_args(argv)
    if a.run == "rg":
        for f in a.f:
            for th in a.theta:
                print(json.dumps(run_polyelectrolyte(f, a.steps, a.equil, a.every, a.prec, a.kappa, theta=th,
                                                     valency=a.valency)), flush=True)
    else:
        print(json.dumps(run_electrolyte_rdf(a.steps, a.equil, max(a.every, 200), a.prec, a.kappa)), flush=True)


if __name__ == "__main__":
    main()
