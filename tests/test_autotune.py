"""The autotuner's host logic: candidate launch shapes come from the plan's own
validation, the fastest measured one is kept and cached, and cache lookups need
no timing. The device timing is replaced by a cost model here; CPU only."""
import json

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import autotune, enuf
    return autotune, enuf


BASE = dict(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4)


def _q(n=1000, charged=100):
    q = np.zeros(n)
    q[:charged // 2] = 1.0
    q[charged // 2:charged] = -1.0
    return q


def test_candidates_are_the_legal_tiles(mods):
    A, E = mods
    # n = 96: the divisors of n in [p, 24]; FP32 grids with n <= 112 also try the five-pass
    # FFT, and the Stockham stages against the two-factor kernels (radix 1 and 2 agree
    # below n = 128)
    c32 = A.candidates(E.make_params(prec="fp32", **BASE), 81000)
    assert sorted({c["tile"] for c in c32}) == [4, 6, 8, 12, 16, 24]
    assert {c["fft_path"] for c in c32} == {0, 1} and len(c32) == 24
    assert {c["fft_radix"] for c in c32} == {0, 2}
    c64 = A.candidates(E.make_params(prec="fp64", **BASE), 81000)
    assert sorted(c["tile"] for c in c64) == [4, 6, 8, 12, 16, 24]
    assert {c["fft_path"] for c in c64} == {0}
    # n = 160: tile 4 would make 40^3 tiles, beyond the binning histogram's 32768
    big = dict(BASE, L=50.0, M=80)
    c = A.candidates(E.make_params(prec="fp32", **big), 375000)
    assert sorted({x["tile"] for x in c}) == [5, 8, 10, 16, 20]
    # from n = 128 on, FP32 also tries radices 2, 3, 4, 5, 8 only against the composite
    # schedule, both against the two-factor kernels
    assert {x["fft_path"] for x in c} == {0} and {x["fft_radix"] for x in c} == {0, 1, 2} and len(c) == 15
    c = A.candidates(E.make_params(prec="fp64", **big), 375000)
    assert {x["fft_radix"] for x in c} == {0} and len(c) == 5
    # n = 512: only tile 16 keeps the histogram within 32768 tiles, and the composite
    # schedule saves no stage there (16 16 2 against 8 8 8), so one candidate remains
    c = A.candidates(E.make_params(prec="fp32", **dict(BASE, L=160.0, M=256)), 1000)
    assert c == [{"tile": 16, "fft_path": 0, "fft_radix": 0}]
    # a wider window raises the smallest tile
    assert min(x["tile"] for x in A.candidates(E.make_params(prec="fp64", **dict(BASE, p=7)), 100)) == 8
    # every candidate is accepted by the plan's validation, every other tile rejected
    p32 = E.make_params(prec="fp32", **BASE)
    for T in range(1, 49):
        try:
            E.enuf_footprint(A._copy(p32, tile=T), 81000)
            ok = True
        except E.EnufError:
            ok = False
        assert ok == (T in {x["tile"] for x in c32}), T


def test_tune_keeps_the_fastest_and_caches_it(mods, tmp_path):
    A, E = mods
    params = E.make_params(prec="fp32", **BASE)
    calls = []

    def cost(p, n_max, pos, q):
        calls.append((p.tile, p.fft_path))
        # fastest: tile 8, fused FFT, two-factor kernels
        return abs(p.tile - 8) + 0.5 * p.fft_path + 0.25 * p.fft_radix + 1.0

    cache = A.TuneCache(str(tmp_path / "tune.json"))
    q = _q()
    r = A.tune(params, 1000, None, q, measure=cost, cache=cache, device="dev")
    assert (r["tile"], r["fft_path"], r["cached"]) == (8, 0, False)
    assert len(calls) == 24 and len(r["timings"]) == 24
    assert params.tile == 0 and params.fft_path == 0          # the caller's params are not modified
    # a second call (and a new cache object on the same file) needs no timing
    calls.clear()
    again = A.tune(params, 1000, None, q, measure=cost, cache=A.TuneCache(cache.path), device="dev")
    assert again["cached"] and (again["tile"], again["fft_path"]) == (8, 0) and not calls
    tp = A.cached_params(params, int((q != 0).sum()), cache=A.TuneCache(cache.path), device="dev")
    assert (tp.tile, tp.fft_path, tp.fft_radix) == (8, 0, 0) and tp.L == params.L and tp.p == params.p
    # force re-measures
    A.tune(params, 1000, None, q, measure=cost, cache=cache, device="dev", force=True)
    assert len(calls) == 24
    with open(cache.path) as f:
        d = json.load(f)
    assert d["version"] == A.CACHE_VERSION and len(d["entries"]) == 1


def test_tuned_params_fill_only_the_launch_choices(mods, tmp_path):
    A, E = mods
    params = E.make_params(prec="fp64", deriv=1, slater_k=1, **BASE)
    tp = A.tuned_params(params, 500, None, _q(500, 50), measure=lambda p, *a: float(p.tile),
                        cache=A.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert tp.tile == 4 and tp.fft_path == 0
    for f in ("L", "alpha", "r_cut", "beta", "kappa", "M", "p", "sigma_s", "kmask", "prec", "deriv", "slater_k"):
        assert getattr(tp, f) == getattr(params, f), f


def test_keys_separate_what_changes_the_kernels(mods):
    A, E = mods
    k = A.cache_key(E.make_params(prec="fp32", **BASE), 100, "dev")
    others = [
        A.cache_key(E.make_params(prec="fp64", **BASE), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", deriv=1, **BASE), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", slater_k=1, **BASE), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", kmask=1, **BASE), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", **dict(BASE, p=5)), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", **dict(BASE, M=64)), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", **dict(BASE, r_cut=4.0)), 100, "dev"),
        A.cache_key(E.make_params(prec="fp32", **BASE), 1000, "dev"),
        A.cache_key(E.make_params(prec="fp32", **BASE), 100, "other"),
    ]
    assert len(set(others + [k])) == len(others) + 1
    # the same shape at another kappa or a charge count in the same power of two shares the entry
    assert A.cache_key(E.make_params(prec="fp32", **dict(BASE, kappa=2.0)), 120, "dev") == k
    # M = 0 keys by the grid rule's M
    assert A.cache_key(E.make_params(prec="fp32", **dict(BASE, M=0)), 100, "dev") == k


def test_a_stale_or_broken_cache_is_ignored(mods, tmp_path):
    A, E = mods
    p = tmp_path / "tune.json"
    p.write_text(json.dumps({"version": A.CACHE_VERSION + 1, "entries": {"x": {"tile": 4}}}))
    assert A.TuneCache(str(p)).entries == {}
    p.write_text("{not json")
    assert A.TuneCache(str(p)).entries == {}
    assert A.TuneCache(str(tmp_path / "absent" / "t.json")).entries == {}


def test_no_legal_tile_is_an_error(mods, tmp_path):
    A, E = mods
    # n = 1000: its divisors in [p, 24] (4, 5, 8, 10, 20) all give more than 32768 tiles
    params = E.make_params(prec="fp32", **dict(BASE, M=500))
    with pytest.raises(E.EnufError) as e:
        A.tune(params, 100, None, _q(100, 10), measure=lambda *a: 1.0,
               cache=A.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert e.value.status == E.ENUF_ERR_UNSUPPORTED


def test_serving_backend_takes_cached_choices(mods, tmp_path):
    """The serving backend looks tuned shapes up in the cache (no timing) and
    leaves untuned shapes and systems that name their tile alone."""
    pytest.importorskip("torch")
    A, E = mods
    from paper_1303_4523_gb300.serving import GpuBackend, Request, SystemSpec
    q = _q(3000, 300)
    spec = SystemSpec("s", 30.0, dict(alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, p=4), np.zeros((3000, 3)), q,
                      M=48)
    req = Request(0, "force", spec, prec="fp32")
    cache = A.TuneCache(str(tmp_path / "t.json"))
    be = GpuBackend(tune_cache=cache)
    assert be._params(req).tile == 0                      # not tuned yet
    key = A.cache_key(E.make_params(prec="fp32", **BASE), 300, A._device_name())
    cache.put(key, {"tile": 8, "fft_path": 1, "fft_radix": 0, "ms": 1.0, "timings": []})
    p = be._params(req)
    assert (p.tile, p.fft_path) == (8, 1)
    assert be.footprint(req) == E.enuf_footprint(p, 3000) + 3000 * 7 * 4
    assert GpuBackend()._params(req).tile == 0            # without a cache
    named = Request(1, "force", SystemSpec("t", 30.0, dict(spec.params, tile=16), spec.pos, q, M=48), prec="fp32")
    assert be._params(named).tile == 16


def test_tune_picks_the_radix_schedule(mods, tmp_path):
    A, E = mods
    params = E.make_params(prec="fp32", **dict(BASE, L=50.0, M=80))    # n = 160
    # a cost model where the plain radices (fft_radix = 1) are fastest
    r = A.tune(params, 1000, None, _q(), measure=lambda p, *a: 2.0 - (p.fft_radix == 1) + 0.01 * p.tile,
               cache=A.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert (r["tile"], r["fft_path"], r["fft_radix"]) == (5, 0, 1)
    tp = A.cached_params(params, 100, cache=A.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert (tp.tile, tp.fft_radix) == (5, 1)


def test_a_failing_candidate_is_skipped(mods, tmp_path):
    A, E = mods
    params = E.make_params(prec="fp64", **BASE)

    def cost(p, *a):
        if p.tile == 4:
            raise E.EnufError(E.ENUF_ERR_OOM, "no room")
        return float(p.tile)

    r = A.tune(params, 1000, None, _q(), measure=cost, cache=A.TuneCache(str(tmp_path / "t.json")), device="dev")
    assert r["tile"] == 6
    failed = [t for t in r["timings"] if t["ms"] is None]
    assert [t["tile"] for t in failed] == [4] and "no room" in failed[0]["error"]

    def broken(p, *a):
        raise E.EnufError(E.ENUF_ERR_OOM, "no room")

    with pytest.raises(E.EnufError):
        A.tune(params, 1000, None, _q(), measure=broken, cache=A.TuneCache(str(tmp_path / "u.json")), device="dev")


def test_batch_candidates_keep_the_launch_sequence(mods, tmp_path):
    """For a batch (sequence=True) the FP32 candidates are the plans a batch runs in
    its one launch sequence: two-factor fused FFT planes, the tile spreading form and
    a column-form tile edge; FP64 batches (one graph branch per system) are unchanged."""
    A, E = mods
    p32 = E.make_params(prec="fp32", **BASE)
    seq = A.candidates(p32, 81000, sequence=True)
    assert seq and all(A._sequence_ok(A._copy(p32, **c), 81000) for c in seq)
    assert sorted({c["tile"] for c in seq}) == [8, 12, 16, 24]
    assert {(c["fft_path"], c["fft_radix"]) for c in seq} == {(0, 0)}
    p64 = E.make_params(prec="fp64", **BASE)
    assert A.candidates(p64, 81000, sequence=True) == A.candidates(p64, 81000)
    # the cost model prefers tile 4 (outside the sequence); a batch tune picks among the rest
    cache = A.TuneCache(str(tmp_path / "t.json"))
    cost = lambda prm, n, pos, q: float(prm.tile)   # noqa: E731
    single = A.tune(p32, 81000, None, _q(), measure=cost, cache=cache, device="dev")
    batch = A.tune(p32, 81000, None, _q(), measure=cost, cache=cache, device="dev", sequence=True)
    assert single["tile"] == 4 and batch["tile"] == 8 and single["key"] != batch["key"]
