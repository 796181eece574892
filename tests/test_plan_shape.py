"""The plan's derived shape from the host logic alone (enuf_plan_shape): grid
rule, tile edge, FFT path and radix schedule, workspace bytes. CPU only."""
import pytest


@pytest.fixture(scope="module")
def enuf():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf as E
    return E


def _shape(enuf, n_max=16, **kw):
    return enuf.plan_shape(enuf.make_params(**kw), n_max)


def _radices(info):
    return list(info.fft_radix[:info.fft_stages])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_radix_schedules(enuf, prec):
    """Stockham stages (fft_radix = 2, FP64's default): fewest stages over
    2, 3, 4, 5, 8; FP32 grids from n = 128 on take the composite radices 6,
    10, 12, 16, 20 when that saves a stage, unless fft_radix = 1."""
    want = {16: [8, 2], 32: [8, 4], 36: [4, 3, 3], 60: [5, 4, 3], 96: [8, 4, 3], 128: [8, 8, 2],
            160: [8, 5, 4], 192: [8, 8, 3], 320: [8, 8, 5], 512: [8, 8, 8]}
    if prec == "fp32":
        want.update({128: [16, 8], 160: [20, 8], 192: [16, 12], 320: [20, 16]})
    for n, rad in want.items():
        kw = dict(prec=prec, L=2.0 * n, alpha=1.0, r_cut=3.0, beta=0.0, kappa=1.0, M=n // 2, p=4)
        info = _shape(enuf, fft_radix=2, **kw)
        assert info.n == n and _radices(info) == rad and not info.fft_two_factor, (n, _radices(info))
        prod = 1
        for r in rad:
            prod *= r
        assert prod == n
        plain = _radices(_shape(enuf, fft_radix=1, **kw))
        assert all(r in (2, 3, 4, 5, 8) for r in plain) and len(plain) >= len(rad)
        if prec == "fp64" or n < 128:
            assert plain == rad


def test_two_factor_split(enuf):
    """FP32 plans with fft_radix = 0 run the two-factor kernels when n = f1 f2
    with both factors in {4, 5, 6, 8, 10, 12, 16, 20}: the most balanced split,
    ties to the larger f2; other n (and FP64) keep the Stockham stages."""
    want = {16: (4, 4), 32: (4, 8), 36: (6, 6), 40: (5, 8), 48: (6, 8), 60: (6, 10), 64: (8, 8),
            72: (6, 12), 80: (8, 10), 96: (8, 12), 100: (10, 10), 128: (8, 16), 160: (10, 16),
            192: (12, 16), 200: (10, 20), 256: (16, 16), 320: (16, 20), 400: (20, 20)}
    for n, (f1, f2) in want.items():
        kw = dict(L=2.0 * n, alpha=1.0, r_cut=3.0, beta=0.0, kappa=1.0, M=n // 2, p=4)
        info = _shape(enuf, prec="fp32", **kw)
        assert info.fft_two_factor == 1 and _radices(info) == [f1, f2], (n, _radices(info))
        assert _shape(enuf, prec="fp64", **kw).fft_two_factor == 0
    for n in (8, 12, 108, 180, 216, 288, 512):   # no split into two of the radices
        kw = dict(L=2.0 * n, alpha=1.0, r_cut=min(3.0, n), beta=0.0, kappa=1.0, M=n // 2, p=2)
        info = _shape(enuf, prec="fp32", **kw)
        assert info.fft_two_factor == 0 and _radices(info) == _radices(_shape(enuf, prec="fp32", fft_radix=2, **kw))


def test_fft_path(enuf):
    """FP32 grids up to n = 112 run the fused plane passes (3 kernels) unless
    fft_path = 1; FP64 and larger grids run the five line passes."""
    base = dict(alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, p=4)
    for M, L in ((16, 10.0), (48, 30.0), (54, 33.75)):
        assert _shape(enuf, prec="fp32", M=M, L=L, **base).fft_kernels == 3
        assert _shape(enuf, prec="fp32", M=M, L=L, fft_path=1, **base).fft_kernels == 5
        assert _shape(enuf, prec="fp64", M=M, L=L, **base).fft_kernels == 5
    assert _shape(enuf, prec="fp32", M=64, L=40.0, **base).fft_kernels == 5


def test_tile_rule(enuf):
    """Default tile: the smallest divisor of n that is >= p and at least r_c
    wide (so the real-space stencil is 3^3 tiles), within the 24-point limit."""
    base = dict(alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, p=4, prec="fp32")
    cases = [  # (L, M, tile): r_c n / L grid points
        (30.0, 48, 12),   # 9.6 -> 12
        (10.0, 16, 16),   # 9.6 -> 16
        (12.7, 18, 9),    # 8.5 -> 9 (an odd edge)
        (12.5, 20, 10),   # 9.6 -> 10
        (100.0, 160, 10),  # 9.6 -> 10
        (10.0, 32, 8),    # 19.2: no divisor of 64 in [20, 24] -> 8 (smallest >= 8)
    ]
    for L, M, T in cases:
        info = _shape(enuf, L=L, M=M, **base)
        assert info.tile == T, (L, M, info.tile)
        assert info.n % info.tile == 0 and info.n_tiles == (info.n // info.tile) ** 3
    # an explicit tile is kept
    assert _shape(enuf, L=30.0, M=48, tile=8, **base).tile == 8


def test_bytes_agree_with_footprint(enuf):
    for kw in (dict(prec="fp32"), dict(prec="fp64"), dict(prec="fp32", deriv=1), dict(prec="fp64", slater_k=1)):
        params = enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4, **kw)
        assert enuf.plan_shape(params, 81000).device_bytes == enuf.enuf_footprint(params, 81000)
        assert enuf.plan_shape(params, 81000).n_max == 81000
    p32 = enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4, prec="fp32")
    p64 = enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4, prec="fp64")
    assert enuf.plan_shape(p32, 81000).device_bytes < enuf.plan_shape(p64, 81000).device_bytes
    # M = 0: the grid rule's M (1.6 L to the nearest even 2^a 3^b 5^c)
    info = _shape(enuf, L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=0, p=4)
    assert (info.M, info.n, info.n_c) == (48, 96, 23)


def test_invalid_parameters_are_reported(enuf):
    with pytest.raises(enuf.EnufError) as e:
        _shape(enuf, L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=47, p=4)
    assert e.value.status == enuf.ENUF_ERR_INVALID
    with pytest.raises(enuf.EnufError) as e:
        _shape(enuf, L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=14, p=4)
    assert e.value.status == enuf.ENUF_ERR_UNSUPPORTED


@pytest.mark.parametrize("L,M", [(10.0, 16), (20.0, 32), (30.0, 48), (40.0, 64), (50.0, 80), (100.0, 160),
                                 (11.0, 18), (12.5, 20), (15.0, 24)])
def test_grid_rule(enuf, L, M):
    """M = 0: 1.6 L rounded to the nearest even 2^a 3^b 5^c integer (one grid
    point per 0.6 R_c of the base grid; n_c = 7 at L = 10)."""
    info = _shape(enuf, L=L, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=0, p=4)
    assert info.M == M and info.n == 2 * M and info.n_c == M // 2 - 1


def test_real_space_stencil_limit(enuf):
    """A tile narrower than r_c / 5 would make the real-space stencil more
    than 1024 tiles (11^3 here): the plan refuses it as unsupported."""
    base = dict(L=20.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=64, p=4, prec="fp32")
    with pytest.raises(enuf.EnufError) as e:
        _shape(enuf, tile=4, **base)
    assert e.value.status == enuf.ENUF_ERR_UNSUPPORTED
    assert _shape(enuf, tile=8, **base).tile == 8        # 7^3 tiles


def test_scatter_spread_admission(enuf):
    """spread = 4 (the scatter form) is taken where its region rules hold and
    refused otherwise: p != 4, a region of 2 tiles that does not divide the 9
    tiles per axis, a grid too small for a unique window offset (n = 32 <
    2 (16 + 8 + 8)), and FP64."""
    base = dict(L=19.2, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=48, p=4, tile=12, spread=4)
    assert _shape(enuf, prec="fp32", **base).spread == 4          # n = 96, region 24
    assert _shape(enuf, prec="fp32", **dict(base, tile=16)).spread == 4   # region of one tile
    for bad in (dict(p=3), dict(M=54, L=21.6), dict(M=16, L=6.4, tile=8)):
        with pytest.raises(enuf.EnufError):
            _shape(enuf, prec="fp32", **dict(base, **bad))
    with pytest.raises(enuf.EnufError):
        _shape(enuf, prec="fp64", **base)


def test_pair_launch_form(enuf):
    """enuf_params.pairs: 1 two launches, 2 one launch, 0 the measured automatic
    form (one launch in FP32, two in FP64); anything else is rejected."""
    kw = dict(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4)
    assert _shape(enuf, 81000, prec="fp32", **kw).pairs == 2
    assert _shape(enuf, 81000, prec="fp64", **kw).pairs == 1
    for prec in ("fp32", "fp64"):
        for form in (1, 2):
            assert _shape(enuf, 81000, prec=prec, pairs=form, **kw).pairs == form
    for bad in (-1, 3):
        with pytest.raises(enuf.EnufError):
            _shape(enuf, 81000, prec="fp32", pairs=bad, **kw)
