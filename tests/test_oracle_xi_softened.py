"""Pins of the oracle's softened-xi variant: the cutoff argument of Eq. 3 taken
from the softened distance s = sqrt(r^2 + eps^2), as the paper's kernel does
with its one inverse square root per pair (Sec. II-A), instead of r.

Independent pins: at eps = 0 the variant is the default path bit for bit; a
pair at offset d with softening eps equals the (separately pinned) unsoftened
default pair at the offset stretched to length s, scaled by r/s; the term
vanishes exactly once s >= r_cut; a periodic cKDTree neighbour sum; momentum
conservation; central differences of the variant's own direct sum for its
gradient; theta = 0 lists reproduce the direct sum and its gradient.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1211_4406_gb300 import inputs


def g_factored(xi):
    xi = np.asarray(xi, dtype=np.float64)
    lo = 1 - 8 / 5 * xi ** 3 + 8 / 5 * xi ** 5 - xi ** 6 / 2 - 12 / 35 * xi ** 7 + 3 / 20 * xi ** 8
    hi = (2 - xi) ** 5 * (7 * xi ** 3 + 22 * xi ** 2 + 10 * xi + 4) / 140
    return np.where(xi <= 1, lo, np.where(xi < 2, hi, 0.0))


def kdtree_forces_softened(pos, mass, G, eps, rc):
    tree = cKDTree(pos, boxsize=1.0)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d -= np.round(d)
    r2 = np.sum(d * d, axis=1)
    s = np.sqrt(r2 + eps * eps)
    keep = (s < rc) & (r2 > 0)
    i, j, d, s = i[keep], j[keep], d[keep], s[keep]
    f = G * g_factored(2 * s / rc) / s ** 3
    acc = np.zeros_like(pos)
    np.add.at(acc, i, (f * mass[j])[:, None] * d)
    np.add.at(acc, j, -(f * mass[i])[:, None] * d)
    return acc


def rel_err(a, ref):
    num = np.linalg.norm(a - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-6 * np.median(np.linalg.norm(ref, axis=1)))
    return num / den


def test_eps_zero_is_the_default_path():
    pos, mass = inputs.clustered_box(1500, 8, 51)
    G, rc = 1.0, 0.08
    w = inputs.cotangent(1500, 52).astype(np.float64)
    assert np.array_equal(oracle.brute_force(pos, mass, G, 0.0, rc, True),
                          oracle.brute_force(pos, mass, G, 0.0, rc))
    assert np.array_equal(oracle.brute_vjp(pos, mass, G, 0.0, rc, w, True),
                          oracle.brute_vjp(pos, mass, G, 0.0, rc, w))
    t = oracle.OracleTree(pos, mass, 8, 32)
    t.lists(rc, 0.5)
    assert np.array_equal(t.list_forces(G, 0.0, rc, True), t.list_forces(G, 0.0, rc))
    # the list adjoint adds with OpenMP atomics: equal up to their order
    g1, g0 = t.list_vjp(G, 0.0, rc, w, True), t.list_vjp(G, 0.0, rc, w)
    assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max()


def test_pair_equals_plain_pair_at_the_softened_distance():
    """F_soft(d; eps) = F_plain(d s/r; 0) r/s: the same g(2s/r_cut)/s^3 law,
    pointed along d."""
    rng = np.random.default_rng(3)
    rc, G = 0.1, 1.7
    for _ in range(300):
        d = rng.normal(size=3)
        r = rng.uniform(1e-4, rc)
        d *= r / np.linalg.norm(d)
        eps = rng.uniform(0.0, 0.5) * rc
        s = np.hypot(r, eps)
        got = oracle.pair(d, 0.3, G, eps, rc, xi_softened=True)
        if s >= rc:
            assert np.all(got == 0.0)
            continue
        ref = oracle.pair(d * (s / r), 0.3, G, 0.0, rc) * (r / s)
        # measured against the Newtonian scale G m / s^2: near xi = 2 the
        # printed nested form of g cancels, so g itself has no relative bound
        assert np.abs(got - ref).max() <= 1e-13 * G * 0.3 / s ** 2, (got, ref)


def test_cutoff_is_at_the_softened_distance():
    rc, eps = 0.05, 0.01
    r_edge = np.sqrt(rc * rc - eps * eps)
    for r in (r_edge * (1 + 1e-12), 0.5 * (r_edge + rc), rc * (1 - 1e-12)):
        assert r < rc
        assert np.all(oracle.pair([r, 0, 0], 1.0, 1.0, eps, rc, xi_softened=True) == 0.0)
        assert oracle.pair([r, 0, 0], 1.0, 1.0, eps, rc)[0] > 0.0      # the default still pulls
    # 1 % inside, where g ~ 4e-9 stands well above the printed form's rounding
    a = oracle.pair([r_edge * (1 - 1e-2), 0, 0], 1.0, 1.0, eps, rc, xi_softened=True)
    assert a[0] > 0.0 and a[1] == 0.0 and a[2] == 0.0
    # coincident points contribute nothing, softened or not
    assert np.all(oracle.pair([0, 0, 0], 1.0, 1.0, eps, rc, xi_softened=True) == 0.0)
    assert np.all(oracle.pair([0, 0, 0], 1.0, 1.0, 0.0, rc, xi_softened=True) == 0.0)


def test_variant_departs_from_default_by_order_eps2_over_rc2():
    pos, mass = inputs.clustered_box(3000, 20, 53)
    G, rc = 1.0, 0.07
    for eps in (2e-3, 4e-3):
        a0 = oracle.brute_force(pos, mass, G, eps, rc)
        a1 = oracle.brute_force(pos, mass, G, eps, rc, True)
        e = np.sqrt(np.mean(rel_err(a1, a0) ** 2))
        assert 1e-3 * (eps / rc) ** 2 < e < 30 * (eps / rc) ** 2, (eps, e)


def test_brute_force_matches_independent_neighbour_sum():
    pos, mass = inputs.clustered_box(3000, 20, 54)
    mass = mass * np.linspace(0.5, 1.5, mass.size)
    G, eps, rc = 1.3, 4e-3, 0.07
    acc = oracle.brute_force(pos, mass, G, eps, rc, True)
    ref = kdtree_forces_softened(pos, mass, G, eps, rc)
    assert rel_err(acc, ref).max() < 1e-9


def test_momentum_conservation():
    pos, mass = inputs.clustered_box(2000, 10, 55)
    mass = mass * np.linspace(0.2, 2.0, mass.size)
    acc = oracle.brute_force(pos, mass, 1.0, 3e-3, 0.09, True)
    p = (mass[:, None] * acc).sum(0)
    assert np.all(np.abs(p) < 1e-13 * np.abs(mass[:, None] * acc).sum(0))


def test_brute_vjp_matches_central_differences():
    pos, mass = inputs.clustered_box(400, 4, 56)
    G, eps, rc = 1.0, 6e-3, 0.12
    w = inputs.cotangent(400, 57).astype(np.float64)
    grad = oracle.brute_vjp(pos, mass, G, eps, rc, w, True)
    assert not np.array_equal(grad, oracle.brute_vjp(pos, mass, G, eps, rc, w))
    rng = np.random.default_rng(1)
    for _ in range(24):
        k, c = rng.integers(400), rng.integers(3)
        h = 1e-3 * eps
        p, m = pos.copy(), pos.copy()
        p[k, c] += h
        m[k, c] -= h
        fd = (np.sum(w * oracle.brute_force(p, mass, G, eps, rc, True)) -
              np.sum(w * oracle.brute_force(m, mass, G, eps, rc, True))) / (2 * h)
        assert abs(grad[k, c] - fd) <= 1e-6 * max(abs(fd), np.sqrt(np.mean(grad ** 2)))


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_theta_zero_lists_equal_the_direct_sum(kind):
    n = 2000
    if kind == "uniform":
        pos, mass = inputs.uniform_box(n, 58)
    else:
        pos, mass = inputs.clustered_box(n, 12, 58)
    G, eps, rc = 1.0, 3e-3, 0.08
    w = inputs.cotangent(n, 59).astype(np.float64)
    t = oracle.OracleTree(pos, mass, 8, 32)
    t.lists(rc, 0.0)
    a_l = t.list_forces(G, eps, rc, True)
    a_b = oracle.brute_force(pos, mass, G, eps, rc, True)
    assert rel_err(a_l, a_b).max() < 1e-12
    g_l = t.list_vjp(G, eps, rc, w, True)
    g_b = oracle.brute_vjp(pos, mass, G, eps, rc, w, True)
    assert np.abs(g_l - g_b).max() <= 1e-10 * np.abs(g_b).max()
