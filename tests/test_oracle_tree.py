"""Pins of the oracle's keys, octree, monopoles, groups and interaction lists.

Independent pins: bit-by-bit key decoding and numpy's lexsort for the order;
numpy sums/min/max for the monopoles and boxes; structural invariants of the
octree; hand-worked group packings; scipy's periodic cKDTree for the
neighbour sets a theta = 0 list must contain; the direct sum (pinned in
test_oracle_sums) for theta = 0 and theta = 0.5 list forces; central finite
differences for the list gradient.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1211_4406_gb300 import inputs


def np_keys(pos):
    w = pos - np.floor(pos)
    w[w >= 1.0] = 0.0
    q = np.minimum(np.floor(w * 2.0 ** 21), 2.0 ** 21 - 1).astype(np.uint64)
    key = np.zeros(pos.shape[0], dtype=np.uint64)
    for b in range(21):
        for axis, off in ((0, 2), (1, 1), (2, 0)):
            key |= ((q[:, axis] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + off)
    return key


def test_morton_bits():
    assert oracle.morton(1, 0, 0) == 4
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 1
    assert oracle.morton(2, 0, 0) == 32
    assert oracle.morton(2 ** 21 - 1, 2 ** 21 - 1, 2 ** 21 - 1) == 2 ** 63 - 1
    rng = np.random.default_rng(1)
    for _ in range(200):
        q = rng.integers(0, 2 ** 21, size=3)
        k = oracle.morton(*[int(v) for v in q])
        dec = [sum(((k >> (3 * b + off)) & 1) << b for b in range(21)) for off in (2, 1, 0)]
        assert dec == list(q)


def test_key_wrap_edges():
    assert oracle.key_of(1.0, 0.0, 0.0) == 0
    assert oracle.key_of(-1e-20, 0.0, 0.0) == 0          # wraps to 1.0 -> 0.0
    assert oracle.key_of(-0.5, 2.5, 0.0) == oracle.key_of(0.5, 0.5, 0.0)
    top = oracle.key_of(1 - 1e-12, 1 - 1e-12, 1 - 1e-12)
    assert top == 2 ** 63 - 1
    assert oracle.key_of(0.5, 0.0, 0.0) == 4 << (3 * 20)


def build(pos, mass=None, n_leaf=8, n_crit=64):
    t = oracle.OracleTree(pos, mass, n_leaf, n_crit)
    return t, t.export()


def test_sort_order_matches_lexsort():
    pos, mass = inputs.clustered_box(5000, 30, 2)
    pos[:7] = pos[100]                                    # equal keys: ties by index
    _, ex = build(pos, mass)
    k = np_keys(pos)
    order = np.lexsort((np.arange(pos.shape[0]), k))
    assert np.array_equal(ex.perm, order)
    assert np.array_equal(ex.keys, k[order])


def check_tree(pos, mass, ex, n_leaf):
    n = pos.shape[0]
    w = pos - np.floor(pos)
    w[w >= 1.0] = 0.0
    ws, ms = w[ex.perm], mass[ex.perm]
    nn = ex.level.size
    assert ex.level[0] == 0 and ex.first[0] == 0 and ex.count[0] == n
    assert np.all(np.diff(ex.level) >= 0)                 # breadth-first numbering
    for i in range(nn):
        lv, f, c = int(ex.level[i]), int(ex.first[i]), int(ex.count[i])
        keys = ex.keys[f:f + c].astype(object)
        shift = 3 * (21 - lv)
        assert len({int(k) >> shift for k in keys}) == 1  # one cell per node
        leaf = ex.nchild[i] == 0
        assert leaf == (c <= n_leaf or lv == 21)
        if not leaf:
            ch = np.arange(ex.child[i], ex.child[i] + ex.nchild[i])
            assert np.all(ex.parent[ch] == i) and np.all(ex.level[ch] == lv + 1)
            assert ex.first[ch[0]] == f and ex.first[ch[-1]] + ex.count[ch[-1]] == f + c
            assert np.all(ex.first[ch[1:]] == ex.first[ch[:-1]] + ex.count[ch[:-1]])
            octs = [(int(ex.keys[ex.first[k]]) >> (shift - 3)) & 7 for k in ch]
            assert octs == sorted(set(octs))
        sl = slice(f, f + c)
        assert abs(ex.M[i] - ms[sl].sum()) <= 1e-14 * ex.M[i]
        com = (ms[sl, None] * ws[sl]).sum(0) / ms[sl].sum()
        assert np.allclose(ex.com[i], com, rtol=0, atol=2e-14)   # summation order only
        assert np.array_equal(ex.lo[i], ws[sl].min(0)) and np.array_equal(ex.hi[i], ws[sl].max(0))
        assert np.array_equal(ex.cen[i], (ex.lo[i] + ex.hi[i]) * 0.5)
        assert np.array_equal(ex.half[i], (ex.hi[i] - ex.lo[i]) * 0.5)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 9, 64, 65, 700])
def test_tree_structure_small(n):
    pos, mass = inputs.uniform_box(n, 100 + n)
    mass = mass * np.linspace(0.5, 2.0, n)
    _, ex = build(pos, mass)
    check_tree(pos, mass, ex, 8)


def test_tree_structure_clustered():
    pos, mass = inputs.clustered_box(6000, 40, 9)
    _, ex = build(pos, mass, n_leaf=4, n_crit=32)
    check_tree(pos, mass, ex, 4)


def test_coincident_particles_make_deep_leaf():
    pos = np.tile([[0.3, 0.6, 0.9]], (100, 1))
    mass = np.full(100, 0.01)
    t, ex = build(pos, mass, n_leaf=8, n_crit=64)
    check_tree(pos, mass, ex, 8)
    assert ex.level.max() == 21 and ex.level.size == 22
    assert list(ex.gcount) == [100]                     # a big leaf is its own group


def test_empty_box():
    t, ex = build(np.zeros((0, 3)), np.zeros(0))
    assert ex.level.size == 0 and ex.gfirst.size == 0
    assert t.lists(0.1, 0.5) == 0


def octant_box(counts, rng):
    """Particles placed in the eight octants of the unit box, counts[o] each."""
    pts = []
    for o, c in enumerate(counts):
        corner = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1]) * 0.5
        pts.append(corner + 0.05 + 0.4 * rng.random((c, 3)))
    return np.concatenate(pts)


def test_group_packing_hand_examples():
    rng = np.random.default_rng(4)
    # eight small octants of 3: one run S=24, 3 groups of target 8 -> 9, 9, 6
    _, ex = build(octant_box([3] * 8, rng), None, n_leaf=2, n_crit=10)
    assert list(ex.gcount) == [9, 9, 6]
    # a big octant breaks the run; an empty octant does not
    _, ex = build(octant_box([3, 2, 2, 2, 0, 5, 5, 5], rng), None, n_leaf=2, n_crit=10)
    assert list(ex.gcount) == [9, 10, 5]
    _, ex = build(octant_box([12, 2, 2, 2, 0, 5, 5, 5], rng), None, n_leaf=2, n_crit=10)
    assert sum(ex.gcount[:-3]) == 12 and list(ex.gcount[-3:]) == [6, 10, 5]


def check_groups(ex, n, n_crit):
    assert ex.gfirst[0] == 0
    assert np.all(ex.gfirst[1:] == ex.gfirst[:-1] + ex.gcount[:-1])
    assert ex.gfirst[-1] + ex.gcount[-1] == n
    for f, c in zip(ex.gfirst, ex.gcount):
        # the smallest node that contains the group
        cand = np.where((ex.first <= f) & (ex.first + ex.count >= f + c))[0]
        host = cand[np.argmax(ex.level[cand])]
        if c > n_crit:
            assert ex.nchild[host] == 0 and ex.first[host] == f and ex.count[host] == c
            continue
        if host == 0 and ex.count[0] <= n_crit:
            continue
        while host != 0 and ex.first[host] == f and ex.count[host] == c:
            host = ex.parent[host]             # climb single-child chains
        # the group is a union of whole children of one big node
        assert ex.count[host] > n_crit
        ch = np.arange(ex.child[host], ex.child[host] + ex.nchild[host])
        starts, ends = ex.first[ch], ex.first[ch] + ex.count[ch]
        assert f in starts and f + c in ends


def test_groups_partition_and_nesting():
    for n, seed in [(5000, 1), (20000, 2)]:
        pos, mass = inputs.clustered_box(n, 40, seed)
        _, ex = build(pos, mass, 8, 64)
        check_groups(ex, n, 64)
        sizes = ex.gcount
        assert sizes.max() <= 64 and np.mean(sizes) > 20


def periodic_gap2(p, c, h):
    t = p - c
    t -= np.rint(t)
    e = np.maximum(np.abs(t) - h, 0.0)
    return (e * e).sum(axis=-1)


def test_theta_zero_lists_cover_neighbours_and_match_direct_sum():
    pos, mass = inputs.clustered_box(4000, 25, 13)
    G, eps, rc = 1.0, 1e-3, 0.06
    t, _ = build(pos, mass)
    t.lists(rc, 0.0)
    ex = t.export()
    assert np.all(ex.ent >= 0)                            # theta = 0 never accepts
    w = pos - np.floor(pos)
    ws = w[ex.perm]
    kd = cKDTree(ws, boxsize=1.0)
    for g in range(ex.gfirst.size):
        lst = set(ex.ent[ex.loff[g]:ex.loff[g + 1]].tolist())
        f, c = ex.gfirst[g], ex.gcount[g]
        need = set()
        for i in range(f, f + c):
            need.update(kd.query_ball_point(ws[i], rc * (1 - 1e-12)))
        assert need <= lst
        assert np.all(periodic_gap2(ws[list(lst)], ex.gcen[g], ex.ghalf[g]) < rc * rc)
    acc = t.list_forces(G, eps, rc)
    ref = oracle.brute_force(pos, mass, G, eps, rc)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-6 * np.median(np.linalg.norm(ref, axis=1)))
    assert (np.linalg.norm(acc - ref, axis=1) / den).max() < 1e-12


def test_theta_lists_cover_each_source_once():
    pos, mass = inputs.clustered_box(6000, 30, 17)
    rc, theta = 0.05, 0.5
    t, _ = build(pos, mass)
    t.lists(rc, theta)
    ex = t.export()
    w = pos - np.floor(pos)
    ws = w[ex.perm]
    n_nodes_seen = 0
    for g in range(0, ex.gfirst.size, 3):
        e = ex.ent[ex.loff[g]:ex.loff[g + 1]]
        cover = np.zeros(ws.shape[0], dtype=np.int64)
        parts = e[e >= 0]
        cover[parts] += 1
        gf, gc = ex.gfirst[g], ex.gcount[g]
        for nd in (-e[e < 0] - 1):
            n_nodes_seen += 1
            f, c = ex.first[nd], ex.count[nd]
            cover[f:f + c] += 1
            assert f + c <= gf or gf + gc <= f                       # no overlap with the group
            l = 2.0 ** -ex.level[nd]
            d2 = periodic_gap2(ex.cen[nd], ex.gcen[g], ex.ghalf[g] + ex.half[nd])
            assert l * l < theta * theta * d2                        # opening criterion
            t_ = ex.cen[nd] - ex.gcen[g]
            t_ -= np.rint(t_)
            far = np.abs(t_) + ex.half[nd] + ex.ghalf[g]
            assert np.sum(far * far) < rc * rc                       # inside the cutoff
        inside = periodic_gap2(ws, ex.gcen[g], ex.ghalf[g]) < rc * rc
        assert np.all(cover[inside] == 1)                            # each source once
        assert np.all(cover <= 1)
        assert np.all(inside[parts])                                 # no stray particle
    assert n_nodes_seen > 0


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_theta_half_accuracy_vs_direct_sum(kind):
    if kind == "uniform":
        b = inputs.config_box(1)
    else:
        b = inputs.config_box(4, n_override=16 ** 3 * 4)
    acc, _ = oracle.tree_forces(b.pos, b.mass, b.G, b.eps, b.r_cut, b.theta)
    ref = oracle.brute_force(b.pos, b.mass, b.G, b.eps, b.r_cut)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-6 * np.median(np.linalg.norm(ref, axis=1)))
    e = np.linalg.norm(acc - ref, axis=1) / den
    assert np.sqrt(np.mean(e ** 2)) <= 5e-3


def test_list_vjp_theta_zero_equals_direct_vjp():
    pos, mass = inputs.clustered_box(1500, 10, 23)
    mass = mass * np.linspace(0.5, 1.5, mass.size)
    G, eps, rc = 1.0, 1e-3, 0.08
    w = inputs.cotangent(1500, 30).astype(np.float64)
    t, _ = build(pos, mass)
    t.lists(rc, 0.0)
    g1 = t.list_vjp(G, eps, rc, w)
    g0 = oracle.brute_vjp(pos, mass, G, eps, rc, w)
    assert np.abs(g1 - g0).max() <= 1e-10 * np.abs(g0).max()


def test_list_vjp_matches_frozen_central_differences():
    pos, mass = inputs.clustered_box(3000, 15, 29)
    mass = mass * np.linspace(0.5, 1.5, mass.size)
    G, eps, rc, theta = 1.0, 1e-3, 0.07, 0.5
    w = inputs.cotangent(3000, 31).astype(np.float64)
    t, _ = build(pos, mass)
    t.lists(rc, theta)
    grad = t.list_vjp(G, eps, rc, w)
    rng = np.random.default_rng(2)
    rms = np.sqrt(np.mean(grad ** 2))
    for _ in range(16):
        k, c = rng.integers(3000), rng.integers(3)
        vals = []
        for h in (1e-3 * eps, 0.5e-3 * eps):
            p, m = pos.copy(), pos.copy()
            p[k, c] += h
            m[k, c] -= h
            t.refresh(p)
            lp = np.sum(w * t.list_forces(G, eps, rc))
            t.refresh(m)
            lm = np.sum(w * t.list_forces(G, eps, rc))
            vals.append((lp - lm) / (2 * h))
        t.refresh(pos)
        assert abs(vals[0] - vals[1]) <= 1e-6 * max(abs(vals[0]), rms)   # converged
        assert abs(grad[k, c] - vals[0]) <= 1e-5 * max(abs(vals[0]), rms)


def test_group_ranges_partition_the_sums():
    pos, mass = inputs.clustered_box(3000, 15, 41)
    G, eps, rc = 1.0, 1e-3, 0.07
    w = inputs.cotangent(3000, 42).astype(np.float64)
    t, _ = build(pos, mass)
    t.lists(rc, 0.5)
    ng = t.sizes()[2]
    cut = ng // 3
    full = t.list_forces(G, eps, rc)
    parts = t.list_forces_range(0, cut, G, eps, rc) + t.list_forces_range(cut, ng, G, eps, rc)
    assert np.array_equal(full, parts)
    gfull = t.list_vjp(G, eps, rc, w)
    gparts = t.list_vjp_range(0, cut, G, eps, rc, w) + t.list_vjp_range(cut, ng, G, eps, rc, w)
    assert np.allclose(gfull, gparts, rtol=1e-12, atol=1e-12 * np.abs(gfull).max())


def test_leapfrog_adjoint_matches_frozen_central_differences():
    pos, mass = inputs.clustered_box(2000, 10, 51)
    G, eps, rc, theta, dt, steps = 1.0, 2e-3, 0.09, 0.5, 1e-3, 4
    v0 = np.zeros_like(pos)
    w = inputs.cotangent(2000, 52).astype(np.float64)
    _, _, _, trees = oracle.leapfrog(pos, v0, mass, G, eps, rc, theta, dt, steps, keep_trees=True)
    gx, _ = oracle.leapfrog_adjoint(pos, v0, trees, G, eps, rc, dt, steps,
                                    np.zeros_like(pos), np.zeros_like(pos), w)
    rms = np.sqrt(np.mean(gx ** 2))
    rng = np.random.default_rng(5)
    for _ in range(6):
        k, c = rng.integers(2000), rng.integers(3)
        h = 1e-3 * eps
        p, m = pos.copy(), pos.copy()
        p[k, c] += h
        m[k, c] -= h
        lp = np.sum(w * oracle.leapfrog_frozen(p, v0, trees, G, eps, rc, dt, steps)[2])
        lm = np.sum(w * oracle.leapfrog_frozen(m, v0, trees, G, eps, rc, dt, steps)[2])
        fd = (lp - lm) / (2 * h)
        assert abs(gx[k, c] - fd) <= 1e-6 * max(abs(fd), rms)


@pytest.mark.parametrize("theta,rc", [(0.0, 2.3 / 16), (0.5, 0.49)])
def test_lattice_lists_are_translates_of_one_another(theta, rc):
    """On a 16^3 lattice (coordinates multiples of 1/32, so every offset, gap
    and centre of mass is exact) with 2x2x2 leaves as groups, every group is a
    translate of every other: its list, as a set of minimum-image offsets from
    the group centre (particles and node centres of mass), must be the same
    set.  A sign or minimum-image mistake near a face breaks this."""
    side = 16
    pos, mass = inputs.lattice_box(side)
    ot = oracle.OracleTree(pos, mass, 8, 8)
    ot.lists(rc, theta)                               # r_cut^2 is no sum of squares of k/32: no ties
    ex = ot.export()
    assert ex.gfirst.size == side ** 3 // 8 and np.all(ex.gcount == 8)
    sorted_pos = pos[ex.perm]
    ref = None
    for g in range(ex.gfirst.size):
        e = ex.ent[ex.loff[g]:ex.loff[g + 1]]
        src = np.where((e >= 0)[:, None], sorted_pos[np.maximum(e, 0)], ex.com[np.maximum(-e - 1, 0)])
        d = src - ex.gcen[g]
        d -= np.round(d)
        key = np.concatenate([d * 32.0, (e < 0)[:, None]], axis=1)
        key = key[np.lexsort(key.T[::-1])]
        if ref is None:
            ref = key
            # theta = 0 opens every node; at r_cut = 0.49, theta = 0.5 accepts leaves whose
            # gap exceeds 2 l = 0.25 and whose farthest point stays inside r_cut
            assert (theta == 0.0) == bool(np.all(e >= 0))
        else:
            assert key.shape == ref.shape and np.array_equal(key, ref), g


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_count_useful_matches_neighbour_counts(kind):
    """At theta = 0 every source within r_cut of a particle appears once in its
    group's list as a particle, so the useful pairs are the ordered pairs at
    0 < r < r_cut, which a periodic cKDTree counts independently; in the
    softened-xi variant they are the pairs with r^2 + eps^2 < r_cut^2."""
    n, rc, eps = 3000, 0.09, 0.01
    if kind == "uniform":
        pos, mass = inputs.uniform_box(n, 11)
    else:
        pos, mass = inputs.clustered_box(n, 20, 12)
    t = oracle.OracleTree(pos, mass, 8, 48)
    t.lists(rc, 0.0)
    kd = cKDTree(np.mod(pos, 1.0), boxsize=1.0)
    assert t.count_useful(eps, rc) == 2 * len(kd.query_pairs(rc))
    assert t.count_useful(eps, rc, xi_softened=True) == 2 * len(kd.query_pairs(np.sqrt(rc * rc - eps * eps)))
    ex = t.export()
    assert t.count_useful(eps, rc) < int((ex.gcount * np.diff(ex.loff)).sum())


def test_count_useful_brute_force_with_monopoles():
    """theta = 0.5 lists hold monopoles too: a direct count over the exported
    lists (particle entries at their positions, node entries at their centres
    of mass, the particle itself skipped) agrees; every accepted monopole lies
    inside r_cut of every member of its group, so it always counts."""
    pos, mass = inputs.clustered_box(1500, 6, 13)
    rc, eps = 0.12, 0.004
    t = oracle.OracleTree(pos, mass, 4, 16)
    t.lists(rc, 0.5)
    ex = t.export()
    w = np.mod(pos, 1.0)
    w[w >= 1.0] = 0.0
    xs = w[ex.perm]
    n_nodes_entries = 0
    count = 0
    for g in range(ex.gfirst.size):
        ent = ex.ent[ex.loff[g]:ex.loff[g + 1]]
        src = np.where(ent[:, None] >= 0, xs[np.maximum(ent, 0)], ex.com[np.maximum(-ent - 1, 0)])
        for i in range(ex.gfirst[g], ex.gfirst[g] + ex.gcount[g]):
            d = src - xs[i]
            d -= np.rint(d)
            r = np.sqrt((d * d).sum(axis=1))
            keep = (ent != i) & (r > 0) & (r < rc)
            count += int(keep.sum())
            n_nodes_entries += int((ent < 0).sum())
            assert keep[ent < 0].all()
    assert n_nodes_entries > 0
    assert t.count_useful(eps, rc) == count


def test_list_loss_over_groups_is_the_loss_of_their_particles():
    """or_list_loss_groups over a set of groups equals sum w . a over those
    groups' particles from the (pinned) list forces, and over all groups the
    whole loss."""
    pos, mass = inputs.clustered_box(4000, 8, 17)
    rc, eps, G = 0.1, 2e-3, 1.3
    t = oracle.OracleTree(pos, mass, 8, 32)
    t.lists(rc, 0.5)
    ex = t.export()
    w = inputs.cotangent(4000, 5).astype(np.float64)
    acc = t.list_forces(G, eps, rc)
    groups = [3, 17, 0, 40]
    rows = np.concatenate([ex.perm[ex.gfirst[g]:ex.gfirst[g] + ex.gcount[g]] for g in groups])
    want = float(np.sum(w[rows] * acc[rows]))
    assert abs(t.list_loss_groups(groups, G, eps, rc, w) - want) <= 1e-12 * np.abs(w[rows] * acc[rows]).sum()
    everything = t.list_loss_groups(np.arange(ex.gfirst.size), G, eps, rc, w)
    assert abs(everything - float(np.sum(w * acc))) <= 1e-12 * np.abs(w * acc).sum()
