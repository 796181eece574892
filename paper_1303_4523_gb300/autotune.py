"""Autotuner for the launch choices of a plan that leave the method unchanged.

Three plan parameters change which kernels run and how the oversampled grid
is cut, but not what is computed (results agree to rounding):

  tile      the spreading tile edge T (a divisor of n, p <= T <= 24). It sets
            the spreading kernel (column form for T in 8, 10, 12, 16, 20, 24,
            the work-item form otherwise), the binning histogram and the
            real-space cell list, whose stencil is +-ceil(r_c / (T L / n))
            tiles per axis.
  fft_path  FP32 grids with n <= 112 run the FFT as whole z-planes in shared
            memory (x and y passes fused); fft_path = 1 forces the five line
            passes instead.
  fft_radix the line transforms: 0 runs FP32 grids whose n = f1 f2 on the
            two-factor kernels (both DFTs in registers); 2 runs the Stockham
            stages, with composite radices (6, 10, 12, 16, 20) for FP32 grids
            from n = 128 on when that saves a stage; 1 keeps radices
            2, 3, 4, 5, 8.

The library's own host logic (enuf_plan_shape) decides which tiles are legal
and which choices differ, so the candidates never include a launch shape the
plan would reject, nor two that run the same kernels.
Each candidate is timed on the device with CUDA events over repeated
evaluations of the caller's system; the fastest is kept in a JSON cache keyed
by everything that fixes the kernels' shapes and work: device name,
precision, force mode, Slater placement, mode mask, n, p, the real-space
cutoff in grid units and the charged-bead count (in powers of two).

    from paper_1303_4523_gb300 import autotune
    params = autotune.tuned_params(params, n_max, pos, q)   # device tensors

The cache path is $ENUF_TUNE_CACHE, else ~/.cache/enuf_gb300/tune.json.

For a batch (sequence=True) the FP32 candidates are restricted to the plans
a batch can run as one launch sequence over all systems (two-factor fused
FFT planes, the tile spreading form, a column-form tile edge): a faster
single-system choice outside that set takes its system out of the sequence
and costs the batch more than it saves (measured: the 64-system sweep tuned
per system ran as 576 graph launches in 1.62 ms, against 1.33 ms for one
sequence of 11 launches with the default tiles).
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
from typing import Callable

from . import enuf

CACHE_VERSION = 3
MAX_TILE = 24
FUSED_FFT_MAX_N = 112
COMPOSITE_MIN_N = 128
CHOICES = ("tile", "fft_path", "fft_radix")
SEQUENCE_TILES = (8, 10, 12, 16, 20, 24)   # the column spreading form's tile edges


def default_cache_path() -> str:
    return os.environ.get("ENUF_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "enuf_gb300",
                                                             "tune.json")


def _copy(params: enuf.enuf_params, **over) -> enuf.enuf_params:
    p = enuf.enuf_params()
    C.memmove(C.byref(p), C.byref(params), C.sizeof(enuf.enuf_params))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def grid_n(params: enuf.enuf_params) -> int:
    """Oversampled grid edge n = sigma_s M (M from the plan's grid rule when 0)."""
    M = params.M
    if M == 0:
        from .workloads import grid_rule
        M = grid_rule(params.L)
    return params.sigma_s * M


def _shape(params: enuf.enuf_params, n_max: int):
    """(tile, FFT kernels, radix schedule) of the plan, or None if it is rejected."""
    try:
        info = enuf.plan_shape(params, n_max)
    except enuf.EnufError:
        return None
    return info.tile, info.fft_kernels, info.fft_two_factor, tuple(info.fft_radix[:info.fft_stages])


def _sequence_ok(params: enuf.enuf_params, n_max: int) -> bool:
    """Whether a batch can run this plan in its one launch sequence."""
    try:
        info = enuf.plan_shape(params, n_max)
    except enuf.EnufError:
        return False
    return (params.prec == enuf.ENUF_FP32 and info.fft_two_factor == 1 and info.fft_kernels == 3
            and info.spread == 1 and info.tile in SEQUENCE_TILES)


def candidates(params: enuf.enuf_params, n_max: int, sequence: bool = False) -> list[dict]:
    """Every (tile, fft_path, fft_radix) the plan accepts for these
    parameters, one per distinct launch shape: the FFT choices only where
    they select different kernels or radix schedules. sequence: only those a
    batch runs in its one launch sequence, where there are any."""
    n = grid_n(params)
    fp32 = params.prec == enuf.ENUF_FP32
    paths = [0, 1] if fp32 and n <= FUSED_FFT_MAX_N else [0]
    radices = [0, 2, 1] if fp32 else [0]
    out, seen = [], set()
    for T in range(max(1, params.p), MAX_TILE + 1):
        if n % T:
            continue
        for f in paths:
            for r in radices:
                c = {"tile": T, "fft_path": f, "fft_radix": r}
                shape = _shape(_copy(params, **c), n_max)
                if shape is not None and shape not in seen:
                    seen.add(shape)
                    out.append(c)
    if sequence and fp32:
        seq = [c for c in out if _sequence_ok(_copy(params, **c), n_max)]
        if seq:
            return seq
    return out


def cache_key(params: enuf.enuf_params, n_charged: int, device: str = "", sequence: bool = False) -> str:
    n = grid_n(params)
    rc_grid = params.r_cut * n / params.L
    qb = 0 if n_charged <= 0 else int(math.ceil(math.log2(n_charged)))
    prec = "fp32" if params.prec == enuf.ENUF_FP32 else "fp64"
    return (f"{device}|{prec}|deriv{params.deriv}|slater_k{params.slater_k}|kmask{params.kmask}"
            f"|n{n}|p{params.p}|rc{round(rc_grid * 4) / 4:g}|q2^{qb}" + ("|sequence" if sequence else ""))


class TuneCache:
    """A JSON file of tuned choices: {"version": CACHE_VERSION, "entries":
    {key: {"tile", "fft_path", "fft_radix", "ms", "timings"}}}; a file of
    another version is ignored (and replaced on the next put)."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.entries: dict = {}
        try:
            with open(self.path) as f:
                d = json.load(f)
            if d.get("version") == CACHE_VERSION:
                self.entries = dict(d.get("entries", {}))
        except (OSError, ValueError):
            pass

    def get(self, key: str):
        return self.entries.get(key)

    def put(self, key: str, entry: dict):
        self.entries[key] = entry
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"version": CACHE_VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def time_on_device(params: enuf.enuf_params, n_max: int, pos, q, reps: int = 20, warmup: int = 3) -> float:
    """Milliseconds per evaluation of one plan with these parameters: CUDA
    events on the plan's stream around `reps` back-to-back evaluations, after
    `warmup` untimed ones."""
    import torch
    plan = enuf.Plan(params, n_max)
    try:
        F = torch.empty_like(pos)
        for _ in range(warmup):
            plan.energy_forces(pos, q, F, want_energy=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(plan.stream)
        for _ in range(reps):
            plan.energy_forces(pos, q, F, want_energy=False)
        e1.record(plan.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        plan.close()


def _device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except ImportError:
        pass
    return ""


def tune(params: enuf.enuf_params, n_max: int, pos, q, measure: Callable | None = None,
         cache: TuneCache | None = None, device: str | None = None, force: bool = False,
         sequence: bool = False) -> dict:
    """The fastest candidate for this system, from the cache when present
    (sequence: among those a batch runs in its one launch sequence).

    measure(params, n_max, pos, q) -> ms replaces the device timing (tests
    pass a model of the cost). Returns {"tile", "fft_path", "fft_radix",
    "ms", "timings", "key", "cached"}."""
    measure = measure or time_on_device
    cache = cache if cache is not None else TuneCache()
    device = _device_name() if device is None else device
    n_charged = int((q != 0).sum())
    key = cache_key(params, n_charged, device, sequence)
    hit = None if force else cache.get(key)
    if hit is not None:
        return dict(hit, key=key, cached=True)
    cands = candidates(params, n_max, sequence)
    if not cands:
        raise enuf.EnufError(enuf.ENUF_ERR_UNSUPPORTED, "no legal tile for these parameters")
    timings = []
    for c in cands:
        try:
            ms = float(measure(_copy(params, **c), n_max, pos, q))
        except enuf.EnufError as e:      # e.g. no device memory for this shape: skip it
            timings.append(dict(c, ms=None, error=str(e)))
            continue
        timings.append(dict(c, ms=ms))
    done = [t for t in timings if t["ms"] is not None]
    if not done:
        raise enuf.EnufError(enuf.ENUF_ERR_UNSUPPORTED, "every candidate failed: " + timings[0]["error"])
    best = min(done, key=lambda t: t["ms"])
    entry = {k: best[k] for k in CHOICES}
    entry.update(ms=best["ms"], timings=timings)
    cache.put(key, entry)
    return dict(entry, key=key, cached=False)


def tuned_params(params: enuf.enuf_params, n_max: int, pos, q, **kw) -> enuf.enuf_params:
    """A copy of params with the tuned tile edge and FFT choices filled in."""
    r = tune(params, n_max, pos, q, **kw)
    return _copy(params, **{k: r[k] for k in CHOICES})


def cached_params(params: enuf.enuf_params, n_charged: int, cache: TuneCache | None = None,
                  device: str | None = None) -> enuf.enuf_params:
    """A copy of params with a cached choice filled in, or params unchanged
    when this shape was never tuned (no timing runs here)."""
    cache = cache if cache is not None else TuneCache()
    device = _device_name() if device is None else device
    hit = cache.get(cache_key(params, n_charged, device))
    return params if hit is None else _copy(params, **{k: hit[k] for k in CHOICES})
