"""Ewald parameters from a required accuracy (the two conditions of Eq. 29),
host logic only; pinned to the bound the paper deduces in Sec. 5."""
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq29_alpha_min.txt")


@pytest.fixture(scope="module")
def enuf():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf as E
    return E


def _base(enuf, **kw):
    d = dict(L=10.0, alpha=1.0, r_cut=3.0, beta=4.0, kappa=1.0, M=16, p=4)
    d.update(kw)
    return enuf.make_params(**d)


def _smooth(m):
    for f in (2, 3, 5):
        while m % f == 0:
            m //= f
    return m == 1


def test_alpha_bound_of_the_paper(enuf):
    with open(GOLDEN) as f:
        row = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")][0]
    delta, Rc, rc, alpha_paper, dec = float(row[0]), float(row[1]), float(row[2]), float(row[3]), int(row[4])
    out = enuf.accuracy_params(delta, _base(enuf, L=10.0, r_cut=rc))
    # reduced units (R_c = 1) to 1/Angstrom
    assert round(out.alpha / Rc, dec) == alpha_paper


@pytest.mark.parametrize("delta", [1e-3, 1e-4, 1e-6, 1e-10])
@pytest.mark.parametrize("L,rc", [(10.0, 3.0), (30.0, 3.0), (20.0, 4.0), (50.0, 2.5)])
def test_both_conditions_hold_and_are_tight(enuf, delta, L, rc):
    base = _base(enuf, L=L, r_cut=rc)
    out = enuf.accuracy_params(delta, base)
    a = out.alpha
    # real space: erfc(alpha r_c) <= delta, and no smaller alpha satisfies it
    assert math.erfc(a * rc) <= delta * (1 + 1e-9)
    assert math.erfc(a * (1 - 1e-6) * rc) > delta
    # reciprocal space: the largest kept |n| = n_c = M/2 - 1 meets the bound
    nc = out.M // 2 - 1
    assert math.exp(-math.pi ** 2 * nc ** 2 / (a * L) ** 2) <= delta
    # M is the smallest even 2^a 3^b 5^c integer whose n_c meets it
    assert out.M % 2 == 0 and _smooth(out.M)
    for m in range(4, out.M, 2):
        if _smooth(m):
            assert math.exp(-math.pi ** 2 * (m // 2 - 1) ** 2 / (a * L) ** 2) > delta, m
    # the other fields are kept, and the result makes a valid plan
    for f in ("L", "r_cut", "beta", "kappa", "p", "prec", "tile"):
        assert getattr(out, f) == getattr(base, f)
    info = enuf.plan_shape(out, 1000)
    assert info.M == out.M and info.n_c == nc


def test_the_paper_set_misses_its_own_reciprocal_condition(enuf):
    """Sec. 5 keeps n_c = 7 at L = 10 R_c with alpha = 0.20/Angstrom (1.566 per
    R_c): the reciprocal condition of Eq. 29 gives 0.14, not 1e-4; the grid
    the condition asks for at that alpha is larger."""
    a, L = 0.20 * 7.829, 10.0
    assert abs(math.exp(-math.pi ** 2 * 7 ** 2 / (a * L) ** 2) - 0.14) < 0.005
    # at the smallest alpha for r_c = 3 the same accuracy needs n_c >= 9
    out = enuf.accuracy_params(1e-4, _base(enuf, L=L, r_cut=3.0))
    assert out.M // 2 - 1 >= 9


def test_invalid_requests(enuf):
    for delta in (0.0, 1.0, -1e-3, float("nan")):
        with pytest.raises(enuf.EnufError) as e:
            enuf.accuracy_params(delta, _base(enuf))
        assert e.value.status == enuf.ENUF_ERR_INVALID
    with pytest.raises(enuf.EnufError) as e:
        enuf.accuracy_params(1e-4, _base(enuf, r_cut=6.0))      # r_c > L/2
    assert e.value.status == enuf.ENUF_ERR_INVALID
    with pytest.raises(enuf.EnufError) as e:
        enuf.accuracy_params(1e-12, _base(enuf, L=300.0))       # n > 1024
    assert e.value.status == enuf.ENUF_ERR_UNSUPPORTED
