"""Analysis of the validation runs (radius of gyration, radial distribution
functions) against closed forms and identities; CPU only."""
import math
import sys

import numpy as np
import pytest

from paper_1303_4523_gb300 import validation as V


def test_rg_of_a_straight_chain():
    # n beads spaced b on a line: Rg^2 = b^2 (n^2 - 1) / 12
    n, b, L = 48, 0.7, 30.0
    x = np.zeros((n, 3))
    x[:, 0] = 2.0 + b * np.arange(n)
    assert abs(V.radius_of_gyration(x, L) ** 2 - b * b * (n * n - 1) / 12.0) < 1e-12


def test_rg_ignores_periodic_images():
    rng = np.random.default_rng(5)
    L = 10.0
    steps = rng.normal(size=(30, 3))
    x = np.cumsum(0.7 * steps / np.linalg.norm(steps, axis=1, keepdims=True), axis=0)
    rg = V.radius_of_gyration(x, L)
    shifted = np.mod(x + np.array([7.3, -4.1, 9.9]), L)     # wrapped, chain cut by the faces
    imaged = x + L * rng.integers(-2, 3, size=x.shape)       # arbitrary images per bead
    assert abs(V.radius_of_gyration(shifted, L) - rg) < 1e-12
    assert abs(V.radius_of_gyration(imaged, L) - rg) < 1e-12


def _lattice(k, d=1.0):
    g = np.arange(k) * d
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + 0.25, k * d


def test_pair_counts_of_a_simple_cubic_lattice():
    # every site has 6 neighbours at d, 12 at sqrt(2) d, 8 at sqrt(3) d
    x, L = _lattice(10)
    h = V.pair_histogram(x, None, L, 2.0, 40)      # bins of 0.05
    n = x.shape[0]
    assert h[20] == n * 6 / 2                      # [1.00, 1.05)
    assert h[28] == n * 12 / 2                     # [1.40, 1.45) holds sqrt 2
    assert h[34] == n * 8 / 2                      # [1.70, 1.75) holds sqrt 3
    assert h.sum() == n * (6 + 12 + 8) / 2


def test_rdf_of_uniform_points_is_one():
    rng = np.random.default_rng(7)
    L, n, frames = 10.0, 2000, 4
    h = np.zeros(30)
    for _ in range(frames):
        h += V.pair_histogram(rng.uniform(0, L, size=(n, 3)), None, L, 3.0, 30)
    r, g = V.rdf_normalise(h, n, None, L, 3.0, frames)
    sel = r > 0.5
    assert abs(g[sel].mean() - 1.0) < 0.01
    assert np.abs(g[sel] - 1.0).max() < 0.1


def test_cross_counts_add_up():
    rng = np.random.default_rng(9)
    L = 8.0
    a, b = rng.uniform(0, L, size=(300, 3)), rng.uniform(0, L, size=(200, 3))
    both = V.pair_histogram(np.concatenate([a, b]), None, L, 3.0, 20)
    parts = V.pair_histogram(a, None, L, 3.0, 20) + V.pair_histogram(b, None, L, 3.0, 20) + \
        V.pair_histogram(a, b, L, 3.0, 20)
    assert np.array_equal(both, parts)
    # the cross normalisation: uniform sets give g_ab ~ 1
    r, g = V.rdf_normalise(V.pair_histogram(a, b, L, 3.0, 20), 300, 200, L, 3.0)
    assert abs(g[r > 1.0].mean() - 1.0) < 0.05


def test_numpy_fallback_equals_tree(monkeypatch):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(11)
    L = 6.0
    a, b = rng.uniform(0, L, size=(400, 3)), rng.uniform(0, L, size=(150, 3))
    tree = (V.pair_histogram(a, None, L, 2.5, 25), V.pair_histogram(a, b, L, 2.5, 25))
    monkeypatch.setitem(sys.modules, "scipy.spatial", None)
    plain = (V.pair_histogram(a, None, L, 2.5, 25), V.pair_histogram(a, b, L, 2.5, 25))
    assert np.array_equal(tree[0], plain[0]) and np.array_equal(tree[1], plain[1])


def test_block_sem_of_independent_samples():
    rng = np.random.default_rng(13)
    x = rng.normal(0.0, 2.0, size=20000)
    sem = V.block_sem(x, blocks=20)
    assert 0.6 * 2.0 / math.sqrt(x.size) < sem < 1.5 * 2.0 / math.sqrt(x.size)
