"""Pins of the oracle's direct sum of Eq. 2 and of its gradient.

Independent pins: a periodic neighbour search by scipy's cKDTree with the pair
term summed in numpy from the factored closed form of g; momentum
conservation; lattice symmetry; translation invariance; central finite
differences of the direct sum for the analytic gradient.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1211_4406_gb300 import inputs


def g_closed(xi):
    xi = np.asarray(xi, dtype=np.float64)
    lo = 1 - 8 / 5 * xi ** 3 + 8 / 5 * xi ** 5 - xi ** 6 / 2 - 12 / 35 * xi ** 7 + 3 / 20 * xi ** 8
    hi = (2 - xi) ** 5 * (7 * xi ** 3 + 22 * xi ** 2 + 10 * xi + 4) / 140
    return np.where(xi <= 1, lo, np.where(xi < 2, hi, 0.0))


def kdtree_forces(pos, mass, G, eps, rc):
    """Short-range accelerations from a periodic cKDTree neighbour search."""
    tree = cKDTree(pos, boxsize=1.0)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d -= np.round(d)
    r = np.linalg.norm(d, axis=1)
    keep = (r < rc) & (r > 0)
    i, j, d, r = i[keep], j[keep], d[keep], r[keep]
    f = G * g_closed(2 * r / rc) / (r * r + eps * eps) ** 1.5
    acc = np.zeros_like(pos)
    np.add.at(acc, i, (f * mass[j])[:, None] * d)
    np.add.at(acc, j, -(f * mass[i])[:, None] * d)
    return acc


def rel_err(a, ref):
    num = np.linalg.norm(a - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-6 * np.median(np.linalg.norm(ref, axis=1)))
    return num / den


def test_brute_force_matches_independent_neighbour_sum():
    pos, mass = inputs.clustered_box(3000, 20, 11)
    mass = mass * np.linspace(0.5, 1.5, mass.size)
    G, eps, rc = 1.3, 1e-3, 0.07
    acc = oracle.brute_force(pos, mass, G, eps, rc)
    ref = kdtree_forces(pos, mass, G, eps, rc)
    assert rel_err(acc, ref).max() < 1e-9


def test_momentum_conservation():
    pos, mass = inputs.clustered_box(2000, 10, 5)
    mass = mass * np.linspace(0.2, 2.0, mass.size)
    acc = oracle.brute_force(pos, mass, 1.0, 1e-3, 0.09)
    p = (mass[:, None] * acc).sum(0)
    assert np.all(np.abs(p) < 1e-13 * np.abs(mass[:, None] * acc).sum(0))


def test_lattice_has_zero_force():
    pos, mass = inputs.lattice_box(12)
    acc = oracle.brute_force(pos, mass, 1.0, 1e-3, 3.0 / 12)
    scale = 1.0 / 12 ** 3 / (1.0 / 12) ** 2
    assert np.abs(acc).max() < 1e-12 * scale


def test_translation_invariance():
    pos, mass = inputs.uniform_box(1500, 8)
    a0 = oracle.brute_force(pos, mass, 1.0, 2e-3, 0.1)
    shifted = pos + np.array([0.3712, -0.81, 5.25])
    a1 = oracle.brute_force(shifted, mass, 1.0, 2e-3, 0.1)
    # the shifted coordinates themselves round at ~1e-15; tiny net forces magnify it
    assert rel_err(a1, a0).max() < 1e-7


def test_small_n_edge_cases():
    for n in [0, 1]:
        pos = np.random.default_rng(n).random((n, 3))
        acc = oracle.brute_force(pos, np.ones(n), 1.0, 1e-3, 0.1)
        assert acc.shape == (n, 3) and np.all(acc == 0)
    # two particles across the periodic boundary attract through it
    pos = np.array([[0.001, 0.5, 0.5], [0.999, 0.5, 0.5]])
    acc = oracle.brute_force(pos, np.ones(2), 1.0, 0.0, 0.1)
    assert acc[0, 0] < 0 < acc[1, 0]
    assert abs(acc[0, 0] + acc[1, 0]) < 1e-12 * abs(acc[0, 0])
    # coincident particles contribute nothing, even unsoftened
    pos = np.array([[0.2, 0.2, 0.2]] * 3)
    assert np.all(oracle.brute_force(pos, np.ones(3), 1.0, 0.0, 0.1) == 0)


def test_brute_vjp_matches_central_differences():
    pos, mass = inputs.clustered_box(400, 4, 21)
    G, eps, rc = 1.0, 2e-3, 0.12
    w = inputs.cotangent(400, 28).astype(np.float64)
    grad = oracle.brute_vjp(pos, mass, G, eps, rc, w)
    rng = np.random.default_rng(0)
    for _ in range(24):
        k, c = rng.integers(400), rng.integers(3)
        h = 1e-3 * eps
        p, m = pos.copy(), pos.copy()
        p[k, c] += h
        m[k, c] -= h
        fd = (np.sum(w * oracle.brute_force(p, mass, G, eps, rc)) -
              np.sum(w * oracle.brute_force(m, mass, G, eps, rc))) / (2 * h)
        assert abs(grad[k, c] - fd) <= 1e-6 * max(abs(fd), np.sqrt(np.mean(grad ** 2)))


def test_sampled_brute_force_equals_full():
    pos, mass = inputs.clustered_box(1200, 6, 3)
    full = oracle.brute_force(pos, mass, 1.0, 1e-3, 0.1)
    idx = np.array([0, 17, 599, 1199])
    assert np.array_equal(oracle.brute_force_sample(pos, mass, 1.0, 1e-3, 0.1, idx), full[idx])


def test_sampled_brute_vjp_equals_full_rows():
    pos, mass = inputs.clustered_box(900, 5, 13)
    mass = mass * np.linspace(0.5, 1.5, mass.size)
    w = inputs.cotangent(900, 14).astype(np.float64)
    full = oracle.brute_vjp(pos, mass, 1.0, 1e-3, 0.1, w)
    idx = np.array([0, 5, 448, 899])
    assert np.array_equal(oracle.brute_vjp_sample(pos, mass, 1.0, 1e-3, 0.1, w, idx), full[idx])
