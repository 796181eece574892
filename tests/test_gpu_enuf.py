"""GPU parity of the ENUF electrostatics path against the FP64 CPU oracle.

Every comparison calls the CUDA path through the C ABI (libenuf.so via the
ctypes binding) and the oracle on the same seeded inputs. The oracle is the
plain FP64 one for both precisions: an FP32 run hands it the float-rounded
inputs the GPU saw, and every decision (wrap, grid base, pair cutoff) is the
oracle's own FP64 one.

Tolerances (forces: the stated targets of the two paths; energies: derived
from the arithmetic, each component on its own scale):
- forces, relative RMS over all compared beads: FP64 1e-11, FP32 1e-5;
- forces, bead by bead: |F_i - R_i| / max(|R_i|, rms_j |R_j|) below 100x the
  RMS bound, so that a few bad beads cannot hide in the mean;
- E_real, E_recip, E_self + E_neutral: each against its own magnitude, FP64
  1e-12, FP32 1e-6 (pair and mode terms are formed in the working precision
  and summed in FP64; FP32 real-space sums of alternating sign get the scale
  of their absolute terms, which the oracle cannot give, so the FP32 real
  part is bounded by 1e-6 of max(|E_real|, |E_self|));
- E_total against |E_real| + |E_recip| + |E_self + E_neutral|, the scale its
  rounding follows;
- the virial W = sum r.f is a sum of force terms and gets the force bound
  (FP64 1e-11, FP32 1e-5) on the scale |W_real| + |W_recip| + |W_neutral|.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1303_4523_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-11, E=1e-12, stage=1e-12), "fp32": dict(F=1e-5, E=1e-6, stage=1e-5)}


@pytest.fixture(scope="module")
def enuf():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf as e
    return e


def _inputs(prec, pos, q):
    """Inputs as the GPU sees them (float32-rounded for FP32) and as doubles."""
    if prec == "fp32":
        pos = np.asarray(pos, np.float32).astype(np.float64)
        q = np.asarray(q, np.float32).astype(np.float64)
    return np.asarray(pos, np.float64), np.asarray(q, np.float64)


def _gpu(enuf, prec, P, pos, q, n_max=None):
    dt = torch.float32 if prec == "fp32" else torch.float64
    plan = enuf.Plan(enuf.make_params(prec=prec, **P), n_max if n_max is not None else len(q))
    tp = torch.tensor(pos, dtype=dt, device="cuda").reshape(-1, 3).contiguous()
    tq = torch.tensor(q, dtype=dt, device="cuda").contiguous()
    F = torch.full_like(tp, float("nan"))
    E, Wv = plan.energy_forces(tp, tq, F)
    return plan, F.double().cpu().numpy(), E, Wv


def _oparams(P):
    """Oracle parameters: the GPU-only tiling and FFT-path choices do not change the result."""
    return orc.EwaldParams(**{k: v for k, v in P.items()
                              if k not in ("tile", "fft_path", "fft_radix", "spread", "pairs")})


class Ref:
    """The oracle's forces, energies and virial, with the virial's components."""

    def __init__(self, P, pos, q, sample=None):
        Po = _oparams(P)
        Fr, ER = orc.real_space(Po, pos, q, sample)
        Fk, EK, _, _ = orc.recip_enuf(Po, pos, q, sample)
        ES = orc.self_neutral(Po, q)
        self.F = Fr + Fk
        self.E = np.array([ER[0], EK[0], ES[0] + ES[1], ER[0] + EK[0] + ES[0] + ES[1]])
        self.W = ER[1] + EK[1] + ES[2]
        self.Wscale = abs(ER[1]) + abs(EK[1]) + abs(ES[2])


def _rel_rms(F, R):
    den = (R ** 2).sum()
    return math.sqrt(((F - R) ** 2).sum() / den) if den > 0 else math.sqrt((F ** 2).sum())


def _bead_max(F, R):
    """Largest per-bead error |F_i - R_i| / max(|R_i|, rms_j |R_j|) over the charged beads."""
    rn = np.linalg.norm(R, axis=1)
    keep = rn > 0
    if not keep.any():
        return float(np.abs(F).max()) if F.size else 0.0
    rms = math.sqrt((rn[keep] ** 2).mean())
    return float((np.linalg.norm(F - R, axis=1)[keep] / np.maximum(rn[keep], rms)).max())


def _check_energies(prec, E, Wv, ref):
    t = TOL[prec]["E"]
    Er = ref.E
    own = [abs(Er[0]), abs(Er[1]), abs(Er[2])]
    if prec == "fp32":
        own[0] = max(own[0], abs(Er[2]))
    for k in range(3):
        assert abs(E[k] - Er[k]) <= t * own[k], (k, E, Er)
    assert abs(E[3] - Er[3]) <= t * (abs(Er[0]) + abs(Er[1]) + abs(Er[2])), (E, Er)
    assert abs(Wv - ref.W) <= TOL[prec]["F"] * ref.Wscale, (Wv, ref.W, ref.Wscale)


def _check(prec, F, E, Wv, ref, sample=None):
    t = TOL[prec]
    Fc = F if sample is None else F[sample]
    assert np.all(np.isfinite(F))
    assert _rel_rms(Fc, ref.F) < t["F"], _rel_rms(Fc, ref.F)
    assert _bead_max(Fc, ref.F) < 100 * t["F"], _bead_max(Fc, ref.F)
    _check_energies(prec, E, Wv, ref)


def _sys_small(pset):
    s = W.electrolyte_small(pset)
    return dict(L=s.L, M=s.M, **s.params), s.pos, s.q


CASES = {
    # name: (params, N, L, n_charged, seed)
    "paper_set_M16_p2": ("paper", None),
    "bench_set_M16_p4": ("bench", None),
    "radix3_M24_p3": (dict(L=15.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=24, p=3), (3000, 15.0, 600)),
    "radix5_M20_p5_spherical": (dict(L=12.5, alpha=1.1, r_cut=3.0, beta=1.125, kappa=0.8, M=20, p=5, kmask=1),
                                (2500, 12.5, 400)),
    "two_tiles_M8_p4": (dict(L=6.0, alpha=1.2, r_cut=3.0, beta=4.0, kappa=1.0, M=8, p=4), (300, 6.0, 120)),
    "one_tile_M4_p2": (dict(L=6.0, alpha=1.2, r_cut=3.0, beta=0.0, kappa=1.0, M=4, p=2), (100, 6.0, 40)),
    "p8_M32_point_charges": (dict(L=10.0, alpha=1.5, r_cut=5.0, beta=0.0, kappa=1.0, M=32, p=8),
                             (1000, 10.0, 200)),
    "tile12_M36_p6": (dict(L=20.0, alpha=0.8, r_cut=4.0, beta=4.0, kappa=1.1, M=36, p=6, tile=12),
                      (4000, 20.0, 500)),
    # the largest tile edges, two tiles per axis: windows that wrap around the grid
    "tile20_M20_p4": (dict(L=12.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=20, p=4, tile=20),
                      (1500, 12.0, 300)),
    "tile24_M24_p5": (dict(L=14.0, alpha=1.0, r_cut=3.0, beta=2.0, kappa=1.0, M=24, p=5, tile=24),
                      (2000, 14.0, 400)),
    # odd tile edges (work-item spreading; its shared regions stay aligned), one
    # of them the plan's own choice: the smallest divisor of n = 36 at least
    # r_c n / L = 8.5 grid points wide
    "tile9_M18_p4": (dict(L=11.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=18, p=4, tile=9),
                     (3000, 11.0, 400)),
    "default_tile9_M18_p4": (dict(L=12.7, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=18, p=4),
                             (3000, 12.7, 400)),
    "tile5_M20_p5": (dict(L=12.5, alpha=1.1, r_cut=3.0, beta=1.125, kappa=0.8, M=20, p=5, tile=5),
                     (2500, 12.5, 400)),
    "tile15_M30_p3": (dict(L=18.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=30, p=3, tile=15),
                      (4000, 18.0, 400)),
    # grids from n = 128 on: FP32 plans with the composite radices 16, 20, 12
    "radix16_M64_p4": (dict(L=20.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=64, p=4), (2000, 20.0, 400)),
    "radix20_M80_p3": (dict(L=24.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=80, p=3), (2500, 24.0, 400)),
    "radix12_M96_p4": (dict(L=24.0, alpha=1.0, r_cut=3.0, beta=0.0, kappa=1.0, M=96, p=4), (2500, 24.0, 400)),
}


def _case(name):
    spec, shape = CASES[name]
    if isinstance(spec, str):
        return _sys_small(spec)
    N, L, nq = shape
    s = W.electrolyte(N, L, n_charged=nq, seed_offset=50 + len(name))
    return spec, s.pos, s.q


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_energy_forces_parity(enuf, name, prec):
    P, pos, q = _case(name)
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    _check(prec, F, E, Wv, Ref(P, pos, q))
    # uncharged beads get exactly zero force
    assert np.all(F[q == 0] == 0.0)
    plan.close()


def test_default_tile_can_be_odd(enuf):
    """The plan's own tile choice at n = 36, r_c n / L = 8.5: T = 9."""
    P, _, _ = _case("default_tile9_M18_p4")
    for prec in ("fp32", "fp64"):
        plan = enuf.Plan(enuf.make_params(prec=prec, **P), 100)
        assert (plan.info.n, plan.info.tile, plan.info.n_tiles) == (36, 9, 64)
        plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_stage_plans(enuf, prec):
    """The Stockham stages' radix plans (fft_radix = 2): 2, 3, 4, 5, 8 (greedy
    order), and in FP32 from n = 128 on the two-stage plans with the composite
    radices."""
    want = {16: [8, 2], 32: [8, 4], 96: [8, 4, 3], 128: [8, 8, 2], 160: [8, 5, 4], 192: [8, 8, 3]}
    if prec == "fp32":
        want.update({128: [16, 8], 160: [20, 8], 192: [16, 12]})
    for n, rad in want.items():
        plan = enuf.Plan(enuf.make_params(prec=prec, L=2.0 * n, alpha=1.0, r_cut=3.0, beta=0.0, kappa=1.0,
                                          M=n // 2, p=4, fft_radix=2), 16)
        info = plan.info
        assert list(info.fft_radix[:info.fft_stages]) == rad, (n, list(info.fft_radix[:info.fft_stages]))
        plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("deriv", [0, 1])
def test_five_pass_fft_parity(enuf, name, prec, deriv):
    """The five line passes (the path of grids whose z-planes do not fit in
    shared memory), forced on the small cases, in both force modes."""
    P, pos, q = _case(name)
    P = dict(P, fft_path=1, deriv=deriv)
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    # five line passes, or four when the spreading kernel does the x pass
    assert plan.info.fft_kernels == (4 if plan.info.spread == 3 else 5)
    _check(prec, F, E, Wv, Ref(P, pos, q))
    plan.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("fft_path", [0, 1])
def test_fp32_stockham_parity(enuf, name, fft_path):
    """FP32 on the Stockham stages (fft_radix = 2) instead of the two-factor
    kernels, fused plane passes where they apply and the five line passes."""
    P, pos, q = _case(name)
    P = dict(P, fft_radix=2, fft_path=fft_path)
    pos, q = _inputs("fp32", pos, q)
    plan, F, E, Wv = _gpu(enuf, "fp32", P, pos, q)
    assert plan.info.fft_two_factor == 0
    _check("fp32", F, E, Wv, Ref(P, pos, q))
    plan.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("form", [1, 2, 3])
def test_fp32_spread_forms_parity(enuf, name, form):
    """FP32 spreading forms on the five-pass FFT: the tile form (1), footprint
    bricks written to the grid (2) and bricks fused with the forward x pass
    (3, where the two-factor kernels run and the tile edge is even)."""
    P, pos, q = _case(name)
    P = dict(P, fft_path=1, spread=form)
    pos, q = _inputs("fp32", pos, q)
    shape = enuf.plan_shape(enuf.make_params(prec="fp32", **P), len(q)) if form != 3 else None
    if form == 3:
        # the fused form needs the two-factor kernels, an even tile and a brick of
        # T^2 rows of n points plus >= 2 line pairs of the x transform in 200 KB
        probe = enuf.plan_shape(enuf.make_params(prec="fp32", **dict(P, spread=2)), len(q))
        n, T = probe.n, probe.tile
        f1, f2 = probe.fft_radix[0], probe.fft_radix[1]
        lp = min(16, T * T // 2, (200 * 1024 - T * T * n * 4 - 8 * n) // ((f1 * (f2 + 1) + n + 1) * 8))
        if not (probe.fft_two_factor and T % 2 == 0 and lp >= 2):
            with pytest.raises(enuf.EnufError):
                enuf.plan_shape(enuf.make_params(prec="fp32", **P), len(q))
            return
    plan, F, E, Wv = _gpu(enuf, "fp32", P, pos, q)
    assert plan.info.spread == form and (form == 1 or plan.info.brick_x % plan.info.tile == 0)
    assert shape is None or shape.spread == form
    _check("fp32", F, E, Wv, Ref(P, pos, q))
    if form == 2:   # the grid itself against the oracle's spread grid
        grid = plan.debug_buffer(enuf.ENUF_BUF_GRID).astype(np.float64)
        _, _, g_ref, _ = orc.recip_enuf(_oparams(P), pos, q, want_grid=True)
        assert np.abs(grid - g_ref).max() < TOL["fp32"]["stage"] * np.abs(g_ref).max()
    plan.close()


# the scatter spreading form (spread = 4): p = 4, regions of 2^3 tiles for
# T = 8, 10, 12 and of one tile for T = 16, 20, 24; (M, T), n = 2M
SC_CASES = {"n128_T8_E16": (64, 8), "n160_T10_E20": (80, 10), "n144_T12_E24": (72, 12),
            "n128_T16_E16": (64, 16), "n160_T20_E20": (80, 20), "n144_T24_E24": (72, 24)}


def _sc_inputs(layout, L, seed):
    """uniform: 3000 beads, 1200 charged; clustered: 1500 of the charged beads
    packed into a cube of edge L/5 across the periodic corner (bins of tens of
    beads, several 32-bead chunks each, many atomics on the same points);
    sparse: 7 charged beads (most regions receive none)."""
    rng = np.random.default_rng(seed)
    if layout == "sparse":
        pos = rng.uniform(0.0, L, (400, 3))
        q = np.zeros(400)
        q[:7] = [1.0, -1.0, 2.0, -2.0, 1.0, -0.5, -0.5]
        return pos, q
    n, nq = (3000, 1200) if layout == "uniform" else (3000, 2000)
    pos = rng.uniform(0.0, L, (n, 3))
    if layout == "clustered":
        pos[:1500] = np.mod(rng.uniform(-0.1 * L, 0.1 * L, (1500, 3)), L)
    q = np.zeros(n)
    q[:nq] = np.where(np.arange(nq) % 2 == 0, 1.0, -1.0)
    return pos, q


@pytest.mark.parametrize("name", list(SC_CASES))
@pytest.mark.parametrize("layout", ["uniform", "clustered", "sparse"])
def test_fp32_scatter_spread_parity(enuf, name, layout):
    """The scatter form's grid against the oracle's spread grid, and the
    forces and energies of the evaluation on it, for every region edge."""
    M, T = SC_CASES[name]
    L = 0.2 * M
    P = dict(L=L, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=M, p=4, tile=T, spread=4)
    pos, q = _inputs("fp32", *_sc_inputs(layout, L, 7 + M + T))
    plan, F, E, Wv = _gpu(enuf, "fp32", P, pos, q)
    assert plan.info.spread == 4 and plan.info.tile == T
    grid = plan.debug_buffer(enuf.ENUF_BUF_GRID).astype(np.float64)
    _, _, g_ref, _ = orc.recip_enuf(_oparams(P), pos, q, want_grid=True)
    assert np.abs(grid - g_ref).max() < TOL["fp32"]["stage"] * np.abs(g_ref).max()
    _check("fp32", F, E, Wv, Ref(P, pos, q))
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_gradient_mode_parity(enuf, name, prec):
    """Gradient-mode reciprocal forces (one inverse transform, derivative of the
    window in the gather) against the oracle's gradient mode."""
    P, pos, q = _case(name)
    P = dict(P, deriv=1)
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    _check(prec, F, E, Wv, Ref(P, pos, q))
    assert np.all(F[q == 0] == 0.0)
    h = plan.debug_buffer(enuf.ENUF_BUF_FIELD)
    assert h.shape[0] == 1
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_mode_field_matches_oracle(enuf, prec):
    P, pos, q = _sys_small("bench")
    P = dict(P, deriv=1)
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    h = plan.debug_buffer(enuf.ENUF_BUF_FIELD).astype(np.float64)
    _, _, _, h_ref = orc.recip_enuf(_oparams(P), pos, q, want_h=True)
    t = TOL[prec]["stage"]
    assert np.abs(h - h_ref).max() < 10 * t * np.abs(h_ref).max()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spread_grid_and_fields_match_oracle(enuf, prec):
    """Stage parity: the spread grid (Eq. 14, first half) and the three
    conjugated-NFFT fields before the gather (Eq. 25)."""
    P, pos, q = _sys_small("bench")
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    grid = plan.debug_buffer(enuf.ENUF_BUF_GRID).astype(np.float64)
    h = plan.debug_buffer(enuf.ENUF_BUF_FIELD).astype(np.float64)
    Po = _oparams(P)
    _, _, g_ref, h_ref = orc.recip_enuf(Po, pos, q, want_grid=True, want_h=True)
    t = TOL[prec]["stage"]
    assert np.abs(grid - g_ref).max() < t * np.abs(g_ref).max()
    assert np.abs(h - h_ref).max() < 10 * t * np.abs(h_ref).max()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_cases(enuf, prec):
    P = dict(L=8.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=4)
    rng = np.random.default_rng(4)
    # (a) no beads at all
    plan = enuf.Plan(enuf.make_params(prec=prec, **P), 10)
    dt = torch.float32 if prec == "fp32" else torch.float64
    e = torch.empty((0, 3), dtype=dt, device="cuda")
    E, Wv = plan.energy_forces(e, torch.empty(0, dtype=dt, device="cuda"), torch.empty_like(e))
    assert np.all(E == 0.0) and Wv == 0.0
    plan.close()
    # (b) all uncharged, (c) a single charge, (d) net charge with positions
    # far outside the box, (e) fewer beads than the plan's capacity
    pos = rng.uniform(-20, 30, (257, 3))
    cases = [np.zeros(257), np.eye(1, 257, 100)[0] * 2.0,
             np.where(rng.uniform(size=257) < 0.3, rng.choice([-1.0, 1.0, 2.0], 257), 0.0)]
    for qq in cases:
        p_, q_ = _inputs(prec, pos, qq)
        plan, F, E, Wv = _gpu(enuf, prec, P, p_, q_, n_max=1000)
        ref = Ref(P, p_, q_)
        if np.all(qq == 0):
            assert np.all(F == 0.0) and np.all(E == 0.0)
        elif np.count_nonzero(qq) == 1:
            # a lone charge feels only the NFFT's spurious self-force (exactly 0 in
            # the Ewald sum): compare on the scale of a unit pair force at r = 1
            f0 = P["kappa"] * 4.0
            assert np.abs(F - ref.F).max() < TOL[prec]["F"] * f0 and np.abs(ref.F).max() < 1e-3 * f0
            assert E[0] == 0.0 and ref.E[0] == 0.0
            _check_energies(prec, E, Wv, ref)
        else:
            _check(prec, F, E, Wv, ref)
        plan.close()


def test_n_above_capacity_is_rejected(enuf):
    P = dict(L=8.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=4)
    plan = enuf.Plan(enuf.make_params(**P), 10)
    x = torch.zeros((11, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(enuf.EnufError) as ei:
        plan.energy_forces(x, torch.zeros(11, dtype=torch.float64, device="cuda"), x.clone())
    assert ei.value.status == 1
    plan.close()


def test_repeat_and_pointer_change(enuf):
    """Graph replay gives the same result; new pointers trigger a new capture."""
    P, pos, q = _sys_small("bench")
    plan = enuf.Plan(enuf.make_params(**P), len(q))
    tp = torch.tensor(pos, device="cuda")
    tq = torch.tensor(q, device="cuda")
    F1, F2 = torch.empty_like(tp), torch.empty_like(tp)
    E1, _ = plan.energy_forces(tp, tq, F1)
    E2, _ = plan.energy_forces(tp, tq, F2)
    E3, _ = plan.energy_forces(tp.clone(), tq.clone(), F1)
    assert np.allclose(E1, E2, rtol=1e-14, atol=0) and np.allclose(E1, E3, rtol=1e-14, atol=0)
    assert torch.allclose(F1, F2, rtol=1e-12, atol=1e-14)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_buffer_entry_point(enuf, prec):
    P, pos, q = _sys_small("paper")
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    npd = np.float32 if prec == "fp32" else np.float64
    Fh = np.empty((len(q), 3), npd)
    Eh, Wh = plan.energy_forces_host(pos.astype(npd), q.astype(npd), Fh)
    assert np.allclose(Fh, F, rtol=1e-5 if prec == "fp32" else 1e-12, atol=1e-6 if prec == "fp32" else 1e-13)
    assert np.allclose(Eh, E, rtol=1e-6 if prec == "fp32" else 1e-12)
    plan.close()


def test_stage_timing(enuf):
    P, pos, q = _sys_small("bench")
    plan = enuf.Plan(enuf.make_params(**P), len(q))
    plan.enable_timing(True)
    tp = torch.tensor(pos, device="cuda")
    tq = torch.tensor(q, device="cuda")
    F = torch.empty_like(tp)
    plan.energy_forces(tp, tq, F)
    for st in ("bin", "spread", "fft", "gather", "real", "all"):
        assert plan.stage_time(st) > 0.0
    # binning 2 + window weights, real space, spreading, the FFT kernels, gather (whose
    # last block also reduces the energies)
    assert plan.info.fft_kernels in (3, 5)
    assert plan.launches() == 6 + plan.info.fft_kernels
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_equals_single_plans(enuf, prec):
    systems = [W.electrolyte(N, seed_offset=70 + i) for i, N in enumerate([1500, 3000, 6000, 2000])]
    dt = torch.float32 if prec == "fp32" else torch.float64
    params, pos_l, q_l, F_l, singles, nfft = [], [], [], [], [], []
    for s in systems:
        P = dict(L=s.L, M=s.M, **s.params)
        params.append(enuf.make_params(prec=prec, **P))
        tp = torch.tensor(s.pos, dtype=dt, device="cuda")
        tq = torch.tensor(s.q, dtype=dt, device="cuda")
        pos_l.append(tp)
        q_l.append(tq)
        F_l.append(torch.empty_like(tp))
        pl = enuf.Plan(params[-1], s.N)
        Fs = torch.empty_like(tp)
        Es, _ = pl.energy_forces(tp, tq, Fs)
        singles.append((Fs.double().cpu().numpy(), Es))
        nfft.append(pl.info.fft_kernels)
        pl.close()
    b = enuf.Batch(params, [s.N for s in systems])
    E = b.energy_forces(pos_l, q_l, F_l)
    E2 = b.energy_forces(pos_l, q_l, F_l)
    if prec == "fp32":   # one launch sequence: 8 kernels and one spreading launch per tile edge
        tiles = {enuf.plan_shape(p, s.N).tile for p, s in zip(params, systems)}
        assert b.mode() == 1 and b.launches() == 8 + len(tiles)
    else:                # FP64: one graph branch per system
        assert b.mode() == 0 and b.launches() == sum(6 + k for k in nfft)
    for k, (Fs, Es) in enumerate(singles):
        Fb = F_l[k].double().cpu().numpy()
        tol = 1e-6 if prec == "fp32" else 1e-12
        assert _rel_rms(Fb, Fs) < tol
        assert np.allclose(E[k], Es, rtol=tol) and np.allclose(E2[k], Es, rtol=tol)
    b.close()


def test_batch_sequence_matches_oracle(enuf):
    """The one-launch-sequence batch (FP32): five uneven systems of the batched
    sweep (electrolytes and polyelectrolytes, different boxes, grids and tile
    edges) against the FP64 oracle system by system; then new arrays for two
    systems (the tables are rewritten) and the same results again."""
    systems = W.batch_sweep(5, n_min=3000, n_max=12000)
    params = [enuf.make_params(prec="fp32", L=s.L, M=s.M, **s.params) for s in systems]
    shapes = [enuf.plan_shape(p, s.N) for p, s in zip(params, systems)]
    assert len({sh.n for sh in shapes}) >= 2 and len({sh.tile for sh in shapes}) >= 2
    inputs = [_inputs("fp32", s.pos, s.q) for s in systems]
    pos_l = [torch.tensor(p, dtype=torch.float32, device="cuda") for p, _ in inputs]
    q_l = [torch.tensor(q, dtype=torch.float32, device="cuda") for _, q in inputs]
    F_l = [torch.full_like(p, float("nan")) for p in pos_l]
    b = enuf.Batch(params, [s.N for s in systems])
    assert b.mode() == 1
    E = b.energy_forces(pos_l, q_l, F_l)
    refs = []
    for k, s in enumerate(systems):
        P = dict(L=s.L, M=s.M, **s.params)
        ref = Ref(P, *inputs[k])
        refs.append(ref)
        F = F_l[k].double().cpu().numpy()
        assert np.all(F[inputs[k][1] == 0] == 0.0)
        assert _rel_rms(F, ref.F) < TOL["fp32"]["F"] and _bead_max(F, ref.F) < 100 * TOL["fp32"]["F"], k
        t = TOL["fp32"]["E"]
        Er = ref.E
        assert abs(E[k][1] - Er[1]) <= t * abs(Er[1]) and abs(E[k][2] - Er[2]) <= t * abs(Er[2]), (k, E[k], Er)
        assert abs(E[k][0] - Er[0]) <= t * max(abs(Er[0]), abs(Er[2])), (k, E[k], Er)
        assert abs(E[k][3] - Er[3]) <= t * (abs(Er[0]) + abs(Er[1]) + abs(Er[2])), (k, E[k], Er)
    launches = b.launches()
    # new arrays for systems 1 and 3 (same contents): tables rewritten, graph kept
    pos2 = list(pos_l)
    F2 = list(F_l)
    for k in (1, 3):
        pos2[k] = pos_l[k].clone()
        F2[k] = torch.full_like(F_l[k], float("nan"))
    E2 = b.energy_forces(pos2, q_l, F2)
    assert b.launches() == launches
    for k in range(len(systems)):
        assert _rel_rms(F2[k].double().cpu().numpy(), refs[k].F) < TOL["fp32"]["F"]
        assert np.allclose(E2[k], E[k], rtol=1e-6, atol=1e-6 * abs(refs[k].E[2]))
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["poly81k", "sweep192k"])
def test_full_size_sampled(enuf, prec, which):
    """Full-size systems in the bench's configuration: forces of 256 sampled
    beads against the oracle bead by bead; energies against the full oracle."""
    s = W.polyelectrolyte() if which == "poly81k" else W.electrolyte_sweep(192000)
    P = dict(L=s.L, M=s.M, **s.params)
    pos, q = _inputs(prec, s.pos, s.q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    rng = np.random.default_rng(9)
    ch = np.nonzero(q)[0]
    sample = np.sort(rng.choice(ch, 256, replace=False))
    _check(prec, F, E, Wv, Ref(P, pos, q, sample=sample), sample=sample)
    # properties at any size: the net force vanishes (ik differentiation with
    # a symmetric mode set, real-space pairs in both directions) up to the
    # rounding of the per-bead forces, which adds up like a random walk:
    # |sum F| <= c eps sqrt(N_q) rms|F| with the working precision's eps
    ch = q != 0
    rms = math.sqrt((F[ch] ** 2).sum(1).mean())
    eps = 2.2e-16 if prec == "fp64" else 1.2e-7
    assert np.abs(F.sum(0)).max() < 1e3 * eps * math.sqrt(ch.sum()) * rms, (F.sum(0), rms)
    assert np.all(F[q == 0] == 0.0)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_gradient_mode_sampled(enuf, prec):
    """The 81000-bead polyelectrolyte in gradient mode: 256 sampled forces and
    the energies against the oracle's gradient mode."""
    s = W.polyelectrolyte()
    P = dict(L=s.L, M=s.M, deriv=1, **s.params)
    pos, q = _inputs(prec, s.pos, s.q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    rng = np.random.default_rng(19)
    sample = np.sort(rng.choice(np.nonzero(q)[0], 256, replace=False))
    _check(prec, F, E, Wv, Ref(P, pos, q, sample=sample), sample=sample)
    assert np.all(F[q == 0] == 0.0)
    plan.close()


SLATER_CASES = [n for n in CASES if (CASES[n][0] if isinstance(CASES[n][0], dict) else {"beta": 1.0}).get("beta", 1.0) > 0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", SLATER_CASES)
def test_kspace_slater_parity(enuf, name, prec):
    """Slater form factor in k space with the tabulated real-space kernel
    against the oracle's k-space Slater reading (radial quadrature per pair)."""
    P, pos, q = _case(name)
    P = dict(P, slater_k=1)
    pos, q = _inputs(prec, pos, q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    _check(prec, F, E, Wv, Ref(P, pos, q))
    plan.close()


def test_kspace_slater_needs_beta(enuf):
    with pytest.raises(enuf.EnufError):
        enuf.Plan(enuf.make_params(L=8.0, alpha=1.0, r_cut=3.0, beta=0.0, kappa=1.0, M=16, p=4, slater_k=1), 10)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_kspace_slater_sampled(enuf, prec):
    s = W.polyelectrolyte()
    P = dict(L=s.L, M=s.M, slater_k=1, **s.params)
    pos, q = _inputs(prec, s.pos, s.q)
    plan, F, E, Wv = _gpu(enuf, prec, P, pos, q)
    rng = np.random.default_rng(29)
    sample = np.sort(rng.choice(np.nonzero(q)[0], 128, replace=False))
    _check(prec, F, E, Wv, Ref(P, pos, q, sample=sample), sample=sample)
    plan.close()
