"""Pins of the oracle's ownership and ghost sets for the spatial decomposition
(oracle/domain.py) against independent facts: ownership checked box by box
(every particle in exactly one domain, the one the oracle names); ghost sets
against periodic cKDTree neighbour sets (every particle within r_cut of a
particle of domain d, and not in d, is a ghost of d); the ghost test against
points placed at known periodic distances from a box, across the periodic
boundary and near edges and corners."""
import numpy as np
from scipy.spatial import cKDTree

from oracle import domain as od
from paper_1211_4406_gb300 import inputs


def random_geometry(rng, nx, ny, nz):
    def cuts(m):
        inner = np.sort(rng.uniform(0.05, 0.95, m - 1))
        return np.concatenate([[0.0], inner, [1.0]])
    xc = cuts(nx)
    yc = np.stack([cuts(ny) for _ in range(nx)])
    zc = np.stack([np.stack([cuts(nz) for _ in range(ny)]) for _ in range(nx)])
    return xc, yc, zc


def test_every_particle_has_exactly_its_owner_box():
    rng = np.random.default_rng(3)
    xc, yc, zc = random_geometry(rng, 3, 2, 4)
    pos = rng.uniform(-2.0, 3.0, (4000, 3))
    pos[:5] = [[1.0, 0.5, 0.5], [0.0, 0.0, 0.0], [xc[1], yc[0, 1], 0.3], [-1e-20, 0.2, 0.2], [2.0, 3.0, -4.0]]
    own = od.owner(pos, xc, yc, zc)
    lo, hi = od.boxes(xc, yc, zc)
    w = od.wrap(pos)
    inside = np.all((w[:, None, :] >= lo[None]) & (w[:, None, :] < hi[None]), axis=2)
    assert np.all(inside.sum(axis=1) == 1)
    assert np.array_equal(np.argmax(inside, axis=1), own)
    idx, counts = od.select(pos, xc, yc, zc, "owner")
    assert counts.sum() == pos.shape[0] and np.array_equal(np.sort(idx), np.arange(pos.shape[0]))
    off = np.concatenate([[0], np.cumsum(counts)])
    for d in range(counts.size):
        part = idx[off[d]:off[d + 1]]
        assert np.all(np.diff(part) > 0) and np.all(own[part] == d)


def test_ghost_sets_contain_every_periodic_neighbour():
    rng = np.random.default_rng(5)
    pos, _ = inputs.clustered_box(6000, 12, 5)
    xc, yc, zc = random_geometry(rng, 2, 2, 2)
    rc = 0.07
    own = od.owner(pos, xc, yc, zc)
    kd = cKDTree(od.wrap(pos), boxsize=1.0)
    pairs = kd.query_pairs(rc, output_type="ndarray")
    lo, hi = od.boxes(xc, yc, zc)
    for d in range(8):
        ghosts = set(np.nonzero(od.near(pos, lo[d], hi[d], rc))[0].tolist()) - set(np.nonzero(own == d)[0].tolist())
        a, b = pairs[:, 0], pairs[:, 1]
        need = set(b[(own[a] == d) & (own[b] != d)].tolist()) | set(a[(own[b] == d) & (own[a] != d)].tolist())
        assert need <= ghosts, (d, len(need - ghosts))
        assert len(ghosts) > len(need) > 0          # the box test is a superset of the neighbour test
        idx, counts = od.select(pos, xc, yc, zc, "ghosts", d, rc)
        assert counts[d] == 0
        off = np.concatenate([[0], np.cumsum(counts)])
        for e in range(8):
            part = idx[off[e]:off[e + 1]]
            assert np.all(np.diff(part) > 0)
            assert set(part.tolist()) == set(np.nonzero(od.near(pos, lo[e], hi[e], rc))[0].tolist()) or e == d


def test_ghost_test_at_known_periodic_distances():
    lo = np.array([0.0, 0.3, 0.6])
    hi = np.array([0.25, 0.5, 1.0])
    rc = 0.05
    eps = 1e-9
    pts = []
    want = []
    # across the periodic boundary along x: p = 1 - t is at distance t from x = 0
    for t, inside in [(rc * (1 - eps), True), (rc * (1 + eps), False)]:
        pts.append([1.0 - t, 0.4, 0.8]); want.append(inside)
    # above the box along x and along y
    for t, inside in [(rc * (1 - eps), True), (rc * (1 + eps), False)]:
        pts.append([0.25 + t, 0.4, 0.8]); want.append(inside)
        pts.append([0.1, 0.3 - t, 0.8]); want.append(inside)
    # the box touches z = 1 = 0: a point at z = t is at distance t
    pts.append([0.1, 0.4, 0.02]); want.append(True)
    # near an edge: distance sqrt(2) * a
    a = rc / np.sqrt(2.0)
    for f, inside in [(1 - 1e-6, True), (1 + 1e-6, False)]:
        pts.append([0.25 + a * f, 0.5 + a * f, 0.8]); want.append(inside)
    # near a corner (wrapping in x and z): distance sqrt(3) * b
    b = rc / np.sqrt(3.0)
    for f, inside in [(1 - 1e-6, True), (1 + 1e-6, False)]:
        pts.append([1.0 - b * f, 0.5 + b * f, 0.6 - b * f]); want.append(inside)
    # inside the box, and far away
    pts.append([0.1, 0.4, 0.7]); want.append(True)
    pts.append([0.6, 0.9, 0.3]); want.append(False)
    got = od.near(np.array(pts), lo, hi, rc)
    assert got.tolist() == want
