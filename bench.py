#!/usr/bin/env python3
"""ENUF-DPD force evaluations per second on one polyelectrolyte system.

Workload (synthetic, seeded): 81000 DPD beads in a periodic box L = 30
(density 3); ten chains of 50 beads with harmonic bonds (K = 4, r0 = 0) and
charge fraction 0.5 (q = -1), 250 +1 counterions, 1:1 salt at 0.1 bead
fraction (8100 beads), neutral solvent; a_ij = 25, gamma = 4.5, sigma = 3,
dt = 0.04, lambda = 0.65; electrostatics alpha = 0.975, r_c = 3,
lambda_e = 0.25 (beta = 4), Gamma = 13.87, p = 4, sigma_s = 2, M = 48
(n = 96). One step = one modified velocity-Verlet step of Table 2 with a full
force evaluation: DPD pair + bond forces, real-space erfc + Slater pairs, and
the ENUF reciprocal sum (bin, spread, pruned FFT, convolution, inverse FFT,
gather), plus FP64 totals. The headline is the FP32 path (float arithmetic,
FP64 table and reductions); the FP64 path runs the same workload beside it.

L2 (129 MB) is flushed between timed steps by writing a 256 MB buffer; each
step is timed with CUDA events on the plan's stream.

--impl reference times the FP64 CPU oracle (the only reference there is) on
the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ENUF-DPD force evals/sec at N=81k (FP32 vs FP64, same GPU); p50/p99 latency"
UNIT = "force evals/s"
WORKLOAD = ("polyelectrolyte DPD, N=81000, L=30, 10x50-bead chains f=0.5, 1:1 salt 0.1, "
            "Nq=8600, alpha=0.975, r_c=3, beta=4, Gamma=13.87, p=4, M=48 (n=96); "
            "one Table-2 step with full ENUF+DPD forces per unit")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        return False

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(info, nq, N, esz, nf=3):
    """Algorithmic DRAM bytes of one launch of each kernel group, as the
    scope's measurement section defines them: every array the stage must read
    or write, once, and no intermediate of this design.
      spread : the charged beads (x, y, z, q) read, the n^3 grid written;
      fft    : the grid read (forward), the nf real fields written (inverse),
               and the kept half spectrum of (1 + nf) complex arrays;
      gather : the nf fields and the beads read, the forces written.
    nf: force fields (3 for ik-differentiation, 1 in gradient mode)."""
    n, nc = info.n, info.n_c
    K, nc1 = 2 * nc + 1, nc + 1
    n3 = n ** 3
    modes = nc1 * K * K * 2 * esz
    return {
        "spread": nq * 4 * esz + n3 * esz,
        "gather": nq * 4 * esz + nf * n3 * esz + nq * 3 * esz,
        "fft": n3 * esz + nf * n3 * esz + (1 + nf) * modes,
        "real": nq * 4 * esz * 2 + nq * 3 * esz,
        "dpd": N * (8 * esz) + N * 3 * esz + N * 4,
    }


def fft_pass_bytes(info, esz, nf=3, passes=5):
    """Bytes the five line passes of the FFT read and write between them (the
    spectra after each pass), beside the algorithmic bytes: the overhead of a
    pass-by-pass transform. With the fused plane passes (3 kernels) the
    x/y and inverse y/x intermediates stay in shared memory."""
    n, nc = info.n, info.n_c
    K, nc1 = 2 * nc + 1, nc + 1
    c = 2 * esz
    s1 = n * nc1 * n * c            # after x: [z][kx][y]
    s2 = nc1 * K * n * c            # after y: [kx][ky][z]
    s3 = nf * n * nc1 * K * c       # after z (inverse): [a][z][kx][ky]
    s4 = nf * n * n * nc1 * c       # after inverse y: [a][z][y][kx]
    if passes == 3:
        return 2 * s2 + 2 * s3
    return 2 * s1 + 2 * s2 + 2 * s3 + 2 * s4


def max_over_ranks(dist, totals, device):
    """Timed totals (ms) of this rank -> the maximum over all ranks (the job
    ends when its slowest replica does); identity without a process group."""
    if dist is None:
        return list(totals)
    import torch
    t = torch.tensor(list(totals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world, steps, tot_ms):
    """Whole-job force evaluations per second: every replica ran `steps` steps
    (weak scaling, one system per GPU) within the slowest rank's time."""
    return round(world * 1000.0 * steps / tot_ms, 2)


def run_ours(args, rank, world, dist):
    import torch

    from paper_1303_4523_gb300 import enuf
    from paper_1303_4523_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    s = W.polyelectrolyte()
    dp = W.dpd_params(5)
    P = dict(L=s.L, M=s.M, tile=args.tile, **s.params)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peaks, peak_kind = _peaks()

    def barrier():
        if dist is not None:
            dist.barrier()

    def run_prec(prec, steps, warmup, timing, deriv=0, pairs=0):
        plan = enuf.Plan(enuf.make_params(prec=prec, deriv=deriv, pairs=pairs, **P), s.N)
        sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q,
                              s.bonds, lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"],
                              seed=dp["seed"])
        for _ in range(warmup):
            sysm.step(1)
        torch.cuda.synchronize()
        st = plan.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stage_ms = {k: [] for k in ("spread", "fft", "gather", "real", "dpd", "cell", "bin")}
        barrier()
        torch.cuda.synchronize()
        # the timed steps run the plain step graph (no per-stage event nodes)
        with ClockSampler(dev) as clk:
            t0 = time.perf_counter()
            for k in range(steps):
                with torch.cuda.stream(st):
                    flush.fill_(float(k))
                ev[k][0].record(st)
                sysm.step(1)
                ev[k][1].record(st)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        barrier()
        per = [a.elapsed_time(b) for a, b in ev]
        if timing:   # stage breakdown from a separate pass with per-stage events
            # (with the pairs in one launch the "real" stage is that launch; "dpd" has no event)
            names = [k for k in stage_ms if not (k == "dpd" and plan.info.pairs == 2)]
            plan.enable_timing(True)
            for k in range(min(steps, 20) + 2):
                with torch.cuda.stream(st):
                    flush.fill_(float(k))
                sysm.step(1)
                if k >= 2:
                    for name in names:
                        stage_ms[name].append(plan.stage_time(name))
            plan.enable_timing(False)
        E = sysm.step(0, want_energy=True)
        launches = plan.launches()
        sysm.close()
        plan.close()
        return per, wall, clk.summary(), stage_ms, E, launches

    per32, wall32, clk32, stage32, E32, launches = run_prec("fp32", args.steps, args.warmup, True)
    steps64 = max(3, min(args.steps, 50))
    per64, wall64, clk64, stage64, E64, _ = run_prec("fp64", steps64, args.warmup, False)
    # the same step with gradient-mode reciprocal forces (one inverse transform)
    perg, _, clkg, _, Eg, _ = run_prec("fp32", steps64, args.warmup, False, deriv=1)
    # and with the DPD and real-space pairs as two launches (enuf_params.pairs = 1; the
    # FP32 headline runs them as one): its stage events time the DPD pair kernel in
    # its own launch (the roofline below)
    perp, _, _, stagep, _, launches_p = run_prec("fp32", steps64, args.warmup, True, pairs=1)

    tot32, tot64, totg = max_over_ranks(dist, [sum(per32), sum(per64), sum(perg)], "cuda")
    ms32 = tot32 / args.steps
    ms64 = tot64 / steps64

    # end to end through the public API: host state in (pinned), one step, host state out
    e2e = e2e_run(args, s, dp, P, torch, enuf)

    # roofline of the dominant kernel of the FP32 step (the DPD pair kernel, the
    # largest share of the launch list): ALU-bound, algorithmic work = the pairs
    # within the DPD cutoff x OPS_PER_PAIR lane operations
    plan = enuf.Plan(enuf.make_params(prec="fp32", **P), s.N)
    info = plan.info
    plan.close()
    ab = algorithmic_bytes(info, s.n_charged, s.N, 4)
    means = {k: (sum(v) / len(v) if v else 0.0) for k, v in stage32.items()}
    means_two = {k: (sum(v) / len(v) if v else 0.0) for k, v in stagep.items()}
    means["pairs_fused"] = means["real"]   # the headline's one launch of DPD + real-space pairs
    means["dpd"] = means_two["dpd"]        # k_dpd in its own launch
    means["real"] = means_two["real"]
    npairs, how = dpd_pair_count(s)
    sm_mhz = clk32.get("sm_mhz") or 2070.0
    peak_ops = ALU_LANES * sm_mhz * 1e6 / 1e12
    t_dpd = means["dpd"] * 1e-3
    achieved = npairs * OPS_PER_PAIR / t_dpd / 1e12 if t_dpd > 0 else 0.0
    hbm = {k: {"ms": round(means[k], 5), "GBps": round(ab[k] / (means[k] * 1e-3) / 1e9, 1),
               "frac": round(ab[k] / (means[k] * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
           for k in ("spread", "fft", "gather") if means[k] > 0}
    roof = {"bound": "alu", "kernel": "k_dpd", "achieved": round(achieved, 4), "peak": round(peak_ops, 2),
            "unit": "Tops/s", "frac": round(achieved / peak_ops, 4), "traffic": None,
            "traffic_note": "DRAM bytes are an ncu counter; no capture runs inside the timed bench",
            "peak_kind": f"derived: {ALU_LANES // 128} SMs x 128 lanes x {sm_mhz:.0f} MHz (sampled), 1 op/lane/clock",
            "work": {"pairs": npairs, "pairs_from": how, "ops_per_pair": OPS_PER_PAIR,
                     "algorithmic_bytes": ab["dpd"]},
            "stage_ms": {k: round(v, 5) for k, v in means.items()},
            "hbm_stages": {"peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind, "stages": hbm,
                           "note": "ENUF working set ~35 MB < L2: L2 flushed between steps, intermediates "
                                   "L2-resident; HBM-scale fractions are in --mode sizes"}}

    srt = sorted(per32)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
    s64 = sorted(per64)
    out = {
        "metric": METRIC, "value": job_throughput(world, args.steps, tot32), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms32, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded polyelectrolyte box)",
        "config": {"workload": WORKLOAD, "N": s.N, "n_charged": s.n_charged, "grid_n": info.n,
                   "tile": info.tile, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": round(p50, 5), "p99": round(p99, 5), "mean": round(ms32, 5)},
        "fp64": {"value": job_throughput(world, steps64, tot64), "ms_per_step": round(ms64, 5),
                 "steps": steps64, "p50": round(s64[len(s64) // 2], 5),
                 "p99": round(s64[min(len(s64) - 1, int(math.ceil(0.99 * len(s64))) - 1)], 5),
                 "clocks": clk64},
        "fp32_gradient_mode": {"value": job_throughput(world, len(perg), totg),
                               "ms_per_step": round(totg / len(perg), 5),
                               "p50": round(sorted(perg)[len(perg) // 2], 5), "steps": len(perg),
                               "clocks": clkg,
                               "note": "reciprocal forces as the gradient of the window (deriv = 1)"},
        "fp32_two_pair_launches": {"value": job_throughput(world, len(perp), sum(perp)),
                                   "ms_per_step": round(sum(perp) / len(perp), 5),
                                   "p50": round(sorted(perp)[len(perp) // 2], 5), "steps": len(perp),
                                   "launches_per_step": launches_p,
                                   "note": "DPD and real-space pairs as two launches (pairs = 1); the FP32 "
                                           "headline runs them as one launch (pairs = 0: automatic)"},
        "fp32_over_fp64": round(ms64 / ms32, 2),
        "energies_fp32": [round(x, 6) for x in E32[:8]],
        "energies_fp64": [round(x, 6) for x in E64[:8]],
        "clocks": clk32,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,
        "launches_per_step": launches,
        "roofline": roof,
    }
    return out


def e2e_run(args, s, dp, P, torch, enuf):
    """Same metric through the public API with HOST buffers: each step uploads
    the state (pos, vel, F) from pinned memory, advances one step and reads the
    state and energies back (dpd_step_host: one call, one host synchronisation)."""
    plan = enuf.Plan(enuf.make_params(prec="fp32", **P), s.N)
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q, s.bonds,
                          lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"], seed=dp["seed"])
    pos = torch.empty((s.N, 3), dtype=torch.float32).pin_memory()
    vel = torch.empty((s.N, 3), dtype=torch.float32).pin_memory()
    F = torch.empty((s.N, 3), dtype=torch.float32).pin_memory()
    sysm.get_state_into(pos, vel, F)
    steps = max(3, min(args.steps, 100))
    for k in range(args.warmup + steps):
        if k == args.warmup:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        sysm.step_host(pos, vel, F, 1, want_energy=True)
    dt = time.perf_counter() - t0
    sysm.close()
    plan.close()
    nb = s.N * 3 * 4 * 3
    return {"value": round(steps / dt, 2), "unit": UNIT, "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": nb + 8 * 16, "ms_per_step": round(1000 * dt / steps, 4), "steps": steps}


# DPD pair work: Eq. 3-7 arithmetic (distance, weights, dissipative and random
# terms, forces on both beads) ~40 FP32 operations, plus the Philox4x32-10 draw
# of theta_ij, 10 rounds of 2 wide multiplies, 2 three-way xors and 2 key adds.
OPS_PER_PAIR = 100
ALU_LANES = 152 * 128      # SMs x FP32/INT32 lanes


def dpd_pair_count(s):
    """Pairs within the DPD cutoff 1 in the initial configuration (periodic)."""
    try:
        from scipy.spatial import cKDTree
    except ImportError:
        rho = s.N / s.L ** 3
        return int(round(s.N * rho * 2.0 * math.pi / 3.0)), "estimated N rho 2 pi/3"
    t = cKDTree(np.mod(s.pos, s.L), boxsize=s.L)
    return int(len(t.query_pairs(1.0, output_type="ndarray"))), "counted (k-d tree)"


def cpu_oracle_eval(s, dp, P):
    """One full oracle force evaluation on the host (Table 2 steps 3-5): DPD
    pair + bond forces on every bead, real space and naive ENUF on all charged
    beads. Returns its wall time in seconds."""
    import oracle
    Po = oracle.EwaldParams(**P)
    Do = oracle.DpdParams(**dp)
    every = np.arange(s.N, dtype=np.int32)   # forces of every bead (no O(N^2) energy pass)
    t0 = time.perf_counter()
    Fd, _ = oracle.dpd_forces(Po, Do, s.pos, s.vel, s.types, s.bonds, step=1, sample=every)
    Fe, _, _ = oracle.electrostatics(Po, s.pos, s.q, recip="enuf")
    F = Fd + Fe
    dt = time.perf_counter() - t0
    assert np.isfinite(F).all()
    return dt


def _cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count()


def _timed_evals(steps, budget_s):
    """Up to `steps` full oracle evaluations of the bench workload, stopping
    once `budget_s` seconds have been spent. Returns the per-evaluation times."""
    from paper_1303_4523_gb300 import workloads as W
    s = W.polyelectrolyte()
    dp = W.dpd_params(5)
    P = dict(L=s.L, M=s.M, **s.params)
    times = []
    t0 = time.perf_counter()
    while len(times) < steps and (not times or time.perf_counter() - t0 < budget_s):
        times.append(cpu_oracle_eval(s, dp, P))
    return times, s


def cpu_baseline():
    """The oracle as it stands, timed on the host cores: whole force
    evaluations of the bench workload for about 10-20 s."""
    times, s = _timed_evals(steps=4, budget_s=10.0)
    return {"value": round(len(times) / sum(times), 5), "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{len(times)} full force evaluation(s) of the {s.N}-bead workload (DPD + bonds on all "
                      f"beads, real space + naive ENUF on all {s.n_charged} charged beads), "
                      f"{sum(times):.1f} s"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the only reference there is),
    one full force evaluation per step, on the host cores. The run stops
    after 150 s of timed work; `steps` reports how many ran."""
    budget = 150.0
    if args.warmup:
        _timed_evals(1, 0.0)
    times, s = _timed_evals(args.steps, budget)
    ms = 1000.0 * sum(times) / len(times)
    value = 1000.0 / ms
    srt = sorted(times)
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": 1,
        "steps": len(times), "warmup": min(args.warmup, 1), "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded polyelectrolyte box)",
        "config": {"workload": WORKLOAD, "N": s.N, "n_charged": s.n_charged, "parallelism": "host cores"},
        "latency_ms": {"p50": round(1000 * srt[len(srt) // 2], 2), "p99": round(1000 * srt[-1], 2)},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": f"each step one full force evaluation (DPD + bonds on all {s.N} beads, real "
                                   f"space + naive ENUF on all {s.n_charged} charged beads); {len(times)} of "
                                   f"{args.steps} requested steps within {budget:.0f} s, one warm-up evaluation"},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _stage_roof(plan, info, nq, N, esz, hbm):
    ab = algorithmic_bytes(info, nq, N, esz, 1 if plan.params.deriv else 3)
    out = {}
    for k in ("spread", "fft", "gather"):
        ms = plan.stage_time(k)
        out[k] = {"ms": round(ms, 5), "GBps": round(ab[k] / (ms * 1e-3) / 1e9, 1),
                  "frac": round(ab[k] / (ms * 1e-3) / 1e9 / hbm, 3), "bytes": ab[k]}
    return out


def run_sizes(args):
    """Electrolyte scaling sweep (density 3, 10% charged): one ENUF evaluation
    per size, FP32 and FP64, stage times and HBM fractions; cuFFT (through
    torch.fft) on the same grid timed beside the hand-written FFT."""
    import torch

    from paper_1303_4523_gb300 import enuf
    from paper_1303_4523_gb300 import workloads as W
    peaks, _ = _peaks()
    hbm = peaks["hbm_gbs"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rows = []
    sizes = (3000, 24000, 81000, 192000, 375000, 3000000)
    for N in (sizes if not args.sizes_n else [N for N in sizes if N in args.sizes_n]):
        s = W.electrolyte_sweep(N) if N < 3_000_000 else W.electrolyte(N, seed_offset=499)
        row = {"N": N, "L": round(s.L, 3), "M": s.M}
        variants = (("fp32", "fp32", torch.float32, 4, 0), ("fp64", "fp64", torch.float64, 8, 0),
                    ("fp32_grad", "fp32", torch.float32, 4, 1))
        for key, prec, dt, esz, deriv in (variants[:1] if args.fp32_only else variants):
            P = dict(L=s.L, M=s.M, tile=args.tile, **s.params)
            sp = args.spread if prec == "fp32" else 0
            plan = enuf.Plan(enuf.make_params(prec=prec, deriv=deriv, spread=sp, **P), s.N)
            pos = torch.tensor(s.pos, dtype=dt, device="cuda")
            q = torch.tensor(s.q, dtype=dt, device="cuda")
            F = torch.empty_like(pos)
            for _ in range(3):
                plan.energy_forces(pos, q, F, want_energy=False)
            reps = 20 if N < 1_000_000 else 5
            # the evaluation as it runs (both branches concurrent), CUDA events on its stream
            ev = []
            for _ in range(reps):
                with torch.cuda.stream(plan.stream):
                    flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(plan.stream)
                plan.energy_forces(pos, q, F, want_energy=False)
                b.record(plan.stream)
                ev.append((a, b))
            torch.cuda.synchronize()
            ms_eval = sum(a.elapsed_time(b) for a, b in ev) / reps
            # then the stage breakdown: per-stage events, the branches one after the other
            plan.enable_timing(True)
            for _ in range(2):
                plan.energy_forces(pos, q, F, want_energy=False)
            tot, stages = 0.0, []
            for _ in range(reps):
                with torch.cuda.stream(plan.stream):
                    flush.fill_(1.0)
                plan.energy_forces(pos, q, F, want_energy=False)
                torch.cuda.synchronize()
                tot += plan.stage_time("all")
                stages.append(_stage_roof(plan, plan.info, s.n_charged, s.N, esz, hbm))
            best = {k: min(stages, key=lambda d: d[k]["ms"])[k] for k in ("spread", "fft", "gather")}
            row[key] = {"ms": round(ms_eval, 4), "evals_per_s": round(1000 / ms_eval, 1),
                        "ms_stages_serialized": round(tot / reps, 4), "n": plan.info.n, "stages": best}
            plan.close()
        # cuFFT (torch.fft) on the same grid: R2C forward + 3 C2R inverses, FP32
        n = row["fp32"]["n"]
        g = torch.randn((n, n, n), device="cuda")
        for _ in range(2):
            spec = torch.fft.rfftn(g)
            for _ in range(3):
                torch.fft.irfftn(spec * 1.0001, s=(n, n, n))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(5):
            flush.fill_(2.0)
            e0.record()
            spec = torch.fft.rfftn(g)
            for _ in range(3):
                torch.fft.irfftn(spec * 1.0001, s=(n, n, n))
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        row["cufft_fp32_ms"] = round(min(ts), 4)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr)
    return {"mode": "sizes", "hbm_peak_gbs": hbm, "rows": rows}


def run_batch(args):
    """64 uneven systems (N log-uniform in [3000, 81000], z:1 electrolytes and
    polyelectrolytes) evaluated by one captured graph, against the same plans
    one after another."""
    import torch

    from paper_1303_4523_gb300 import enuf
    from paper_1303_4523_gb300 import workloads as W
    systems = W.batch_sweep(64)
    out = {"mode": "batch", "systems": len(systems), "beads": int(sum(s.N for s in systems))}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        params = [enuf.make_params(prec=prec, L=s.L, M=s.M, **s.params) for s in systems]
        pos = [torch.tensor(s.pos, dtype=dt, device="cuda") for s in systems]
        q = [torch.tensor(s.q, dtype=dt, device="cuda") for s in systems]
        F = [torch.empty_like(p) for p in pos]
        if args.autotune:
            # tile edge and FFT path per system shape, measured once and cached
            from paper_1303_4523_gb300 import autotune
            cache = autotune.TuneCache()
            t0 = time.perf_counter()
            params = [autotune.tuned_params(p, s.N, a, c, cache=cache, sequence=True)
                      for p, s, a, c in zip(params, systems, pos, q)]
            out[prec + "_tune_s"] = round(time.perf_counter() - t0, 2)
            out[prec + "_tiles"] = sorted({p.tile for p in params})
        b = enuf.Batch(params, [s.N for s in systems])
        for _ in range(3):
            b.energy_forces(pos, q, F, want_energy=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(b.stream)
        for _ in range(reps):
            b.energy_forces(pos, q, F, want_energy=False)
        e1.record(b.stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / reps
        launches = b.launches()
        mode = b.mode()
        b.close()
        # aggregate roofline of the ENUF chain: the scope's algorithmic bytes of
        # spreading, FFT and gathering summed over the systems, per graph replay
        esz = 4 if prec == "fp32" else 8
        ab = 0
        for p, sy in zip(params, systems):
            info = enuf.plan_shape(p, sy.N)
            a = algorithmic_bytes(info, sy.n_charged, sy.N, esz)
            ab += a["spread"] + a["fft"] + a["gather"]
        peaks, peak_kind = _peaks()
        plans = [enuf.Plan(p, s.N) for p, s in zip(params, systems)]
        for _ in range(2):
            for pl, a, c, f in zip(plans, pos, q, F):
                pl.energy_forces(a, c, f, want_energy=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            for pl, a, c, f in zip(plans, pos, q, F):
                pl.energy_forces(a, c, f, want_energy=True)
        seq_ms = (time.perf_counter() - t0) * 1000 / 5
        for pl in plans:
            pl.close()
        out[prec] = {"graph_ms": round(ms_batch, 4), "systems_per_s": round(64 * 1000 / ms_batch, 1),
                     "beads_per_s": round(out["beads"] * 1000 / ms_batch, 1), "launches": launches,
                     "one_launch_sequence": bool(mode), "one_by_one_ms": round(seq_ms, 3),
                     "roofline": {"bound": "hbm", "algorithmic_bytes": ab,
                                  "achieved_gbs": round(ab / (ms_batch * 1e-3) / 1e9, 1),
                                  "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
                                  "frac": round(ab / (ms_batch * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                                  "note": "spread + FFT + gather bytes of all systems over the whole "
                                          "evaluation graph (binning and real space included in the time); "
                                          "working set per system L2-resident"}}
    return out


def run_serve(args):
    """Poisson arrivals of ENUF force evaluations (70%) and 10-step DPD blocks
    (30%) on systems of 1e3..1e6 beads plus one 3.0M-bead system, at ~0.8 of
    the measured capacity; continuous batching with admission by HBM
    footprint. Reports p50/p99 latency and aggregate beads*steps/s."""
    import torch

    from paper_1303_4523_gb300.serving import GpuBackend, Server, latency_stats, synthetic_load
    probe = synthetic_load(60, rate_hz=1.0, seed=11)
    be = GpuBackend()
    srv = Server(be, budget_bytes=60 << 30, max_inflight=1)
    for r in probe:
        r.arrival = 0.0
        srv.submit(r)
    t0 = time.perf_counter()
    res = srv.run(realtime=False)
    busy = time.perf_counter() - t0
    mean_service = busy / len(res)
    srv.close()
    rate = 0.8 / mean_service
    reqs = synthetic_load(args.serve_requests, rate_hz=rate, seed=12)
    srv2 = Server(be, budget_bytes=60 << 30, max_inflight=8)
    for r in reqs:
        srv2.submit(r)
    t0 = time.perf_counter()
    res = srv2.run(realtime=True)
    wall = time.perf_counter() - t0
    srv2.close()
    torch.cuda.synchronize()
    st = latency_stats(res)
    bs = sum(r.beads_steps for r in res if r.ok)
    errors = {}
    for r in res:
        if not r.ok:
            key = f"{r.kind}: {r.error[:160]}"
            errors[key] = errors.get(key, 0) + 1
    return {"mode": "serve", "requests": len(res), "rate_hz": round(rate, 1), "wall_s": round(wall, 3),
            "latency": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()},
            "beads_steps_per_s": round(bs / wall, 1), "max_concurrent": srv2.max_concurrent,
            "max_resident_bytes": srv2.max_used, "mean_service_ms_alone": round(1000 * mean_service, 3),
            "errors": errors}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 1000 timed steps after 50 warm-up ones: the p50/p99 latencies of the metric
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="spreading tile edge (0: the plan's choice)")
    ap.add_argument("--mode", default="main", choices=["main", "sizes", "batch", "serve"],
                    help="main: the bench line; sizes/batch/serve: the scaling sweep, the 64-system batch and the "
                         "serving load (each prints its own JSON line)")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--autotune", action="store_true",
                    help="--mode batch: pick each system's tile edge and FFT path by timing them (cached)")
    ap.add_argument("--sizes-n", type=int, nargs="*", default=None,
                    help="--mode sizes: run only these system sizes (of 3000 24000 81000 192000 375000 3000000)")
    ap.add_argument("--spread", type=int, default=0,
                    help="--mode sizes: FP32 spreading kernel (enuf_params.spread: 0 auto, 1 tile form, "
                         "2 footprint bricks, 3 bricks fused with the x pass, 4 scatter form)")
    ap.add_argument("--fp32-only", action="store_true", help="--mode sizes: skip the FP64 and gradient-mode plans")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return

    if args.mode != "main":
        from paper_1303_4523_gb300 import build
        build.build()
        fn = {"sizes": run_sizes, "batch": run_batch, "serve": run_serve}[args.mode]
        print(json.dumps(fn(args)))
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_1303_4523_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    out = run_ours(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
