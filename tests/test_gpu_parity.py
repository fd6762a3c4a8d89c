"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bit-exact: Morton keys, permutation, octree nodes (topology, FP64 monopoles
and boxes), groups and interaction lists.  Within tolerance (written below):
forces on identical lists (FP32 rms <= 1e-6 and max <= 1e-4 relative; FP64
rms <= 1e-8), the adjoint, and theta = 0.5 forces against the direct sum.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300.api import CapturedStep, Params, ShortRangeTree

pytestmark = pytest.mark.gpu

FP32_RMS, FP32_MAX = 1e-6, 1e-4       # FP32 vs FP64 on identical lists
FP64_RMS = 1e-8                      # the oracle's FP64 Eq. 3 form cancels to ~4e-16 near
                                      # xi = 2, which the 1e-6*median guard magnifies
TREE_RMS = 5e-3                       # theta = 0.5 vs the direct sum


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    den = np.maximum(nr, 1e-6 * np.median(nr)) if nr.size else nr
    e = np.linalg.norm(a - ref, axis=1) / den
    return (float(np.sqrt(np.mean(e ** 2))) if e.size else 0.0), (float(e.max()) if e.size else 0.0)


def gpu_tree(box, precision="fp32", theta=None, n_crit=None, n_leaf=None):
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    p = Params(box.G, box.eps, box.r_cut, box.theta if theta is None else theta,
               n_crit or box.n_crit, n_leaf or box.n_leaf, precision)
    return ShortRangeTree(pos, mass, p)


def oracle_tree(box, theta=None, n_crit=None, n_leaf=None):
    t = oracle.OracleTree(box.pos, box.mass, n_leaf or box.n_leaf, n_crit or box.n_crit)
    t.lists(box.r_cut, box.theta if theta is None else theta)
    return t


def assert_structure_equal(gt, ot):
    keys, perm = gt.export_keys()
    ex = ot.export()
    assert np.array_equal(keys, ex.keys)
    assert np.array_equal(perm, ex.perm)
    ints, dbl = gt.export_nodes()
    assert ints.shape[0] == ex.level.size
    oints = np.stack([ex.level, ex.first, ex.count, ex.child, ex.nchild, ex.parent], axis=1)
    assert np.array_equal(ints[:, :6], oints)
    odbl = np.concatenate([ex.M[:, None], ex.com, ex.lo, ex.hi, ex.cen, ex.half], axis=1)
    assert np.array_equal(dbl, odbl)                       # bit-exact FP64 monopoles and boxes
    gi, gd = gt.export_groups()
    assert np.array_equal(gi[:, 0], ex.gfirst) and np.array_equal(gi[:, 1], ex.gcount)
    assert np.array_equal(gd, np.concatenate([ex.gcen, ex.ghalf], axis=1))
    off, ent = gt.export_lists()
    assert np.array_equal(off, ex.loff)
    assert np.array_equal(ent.astype(np.int64), ex.ent)
    return ex


def small_boxes():
    out = []
    for n in [1, 2, 3, 7, 64, 65, 300, 4096]:
        pos, mass = inputs.uniform_box(n, 500 + n)
        out.append(inputs.Box(f"uniform{n}", pos, mass * np.linspace(0.5, 1.5, n), 1.0, 2e-3, 0.2, 0.5))
    pos = np.tile([[0.3, 0.6, 0.9]], (100, 1))
    out.append(inputs.Box("coincident", pos, np.full(100, 0.01), 1.0, 1e-3, 0.1, 0.5))
    pos, mass = inputs.uniform_box(500, 7)
    pos[:, 0] = np.where(pos[:, 0] < 0.5, pos[:, 0] * 0.01, 1 - pos[:, 0] * 0.01)   # hugs x = 0 = 1
    out.append(inputs.Box("wrap", pos, mass, 1.0, 1e-3, 0.15, 0.5))
    pos, mass = inputs.clustered_box(6000, 30, 77)
    out.append(inputs.Box("clustered6k", pos, mass, 1.3, 5e-4, 0.08, 0.5, n_crit=32, n_leaf=4))
    # coordinates at the edges of the integer fast paths of the wrap, the
    # 64-bit images and the 21-bit key digits: zeros of both signs,
    # subnormals, powers of two around 2^-64 and 2^-43, values just below 1
    # and just below 0 (whose wrap rounds to 1 and becomes 0), 1, and values
    # outside [0, 1)
    pos, mass = inputs.uniform_box(600, 11)
    edge = np.array([0.0, -0.0, 5e-324, 2.0 ** -1022, 2.0 ** -1000, 2.0 ** -70, 2.0 ** -65, 2.0 ** -64,
                     2.0 ** -63, 3 * 2.0 ** -64, 2.0 ** -44, 2.0 ** -43, 2.0 ** -21, 0.5, 1 - 2.0 ** -53,
                     1 - 2.0 ** -43, 1 - 2.0 ** -21, 1.0, -2.0 ** -60, -2.0 ** -53, -0.5, 2 - 2.0 ** -52, 3.0,
                     -1e-300, 7.25])
    for c in range(3):
        pos[c * edge.size:(c + 1) * edge.size, c] = edge
        pos[3 * edge.size:4 * edge.size, c] = np.roll(edge, c)
    out.append(inputs.Box("edges", pos, mass, 1.0, 1e-3, 0.15, 0.5))
    return out


@pytest.mark.parametrize("box", small_boxes(), ids=lambda b: b.name)
def test_structure_bit_exact_small(box):
    gt = gpu_tree(box)
    ot = oracle_tree(box)
    assert_structure_equal(gt, ot)
    gt.close()


@pytest.mark.parametrize("box", small_boxes(), ids=lambda b: b.name)
def test_forces_on_identical_lists_small(box):
    ot = oracle_tree(box)
    ref = ot.list_forces(box.G, box.eps, box.r_cut)
    g32 = gpu_tree(box, "fp32")
    a32 = g32.force().double().cpu().numpy()
    g64 = gpu_tree(box, "fp64")
    a64 = g64.force().cpu().numpy()
    if box.n > 1 and np.abs(ref).max() > 0:
        rms32, max32 = rel_err(a32, ref)
        rms64, _ = rel_err(a64, ref)
        # With only a few neighbours inside r_cut a force is one or two terms near
        # the cutoff, where d ln g / d ln r = 5 xi / (2 - xi): FP32's own rounding of r
        # (about 6e-8) then gives ~1e-6 (a correctly rounded FP32 emulation of the
        # 64-particle box gives rms 1.3e-6).  The 1e-6 bound is for the workloads'
        # regime (r_cut = 3 mean spacings, ~110 neighbours); sparse boxes get 1e-5.
        neighbours = box.n * 4.0 / 3.0 * np.pi * box.r_cut ** 3
        rms_bound = FP32_RMS if neighbours >= 10 else 1e-5
        assert rms32 <= rms_bound and max32 <= FP32_MAX, (rms32, max32)
        assert rms64 <= FP64_RMS, rms64
    else:
        assert np.all(a32 == 0) and np.all(a64 == 0)


def test_uniform_32k_structure_and_forces():
    box = inputs.config_box(1)
    gt = gpu_tree(box)
    ot = oracle_tree(box)
    assert_structure_equal(gt, ot)
    ref = ot.list_forces(box.G, box.eps, box.r_cut)
    rms, mx = rel_err(gt.force().double().cpu().numpy(), ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)
    brute = oracle.brute_force(box.pos, box.mass, box.G, box.eps, box.r_cut)
    rms_t, _ = rel_err(gt.force().double().cpu().numpy(), brute)
    assert rms_t <= TREE_RMS
    g64 = gpu_tree(box, "fp64")
    assert rel_err(g64.force().cpu().numpy(), ref)[0] <= FP64_RMS


def test_clustered_262k_structure_forces_and_tree_accuracy():
    box = inputs.config_box(4)
    gt = gpu_tree(box)
    ot = oracle_tree(box)
    assert_structure_equal(gt, ot)
    ref = ot.list_forces(box.G, box.eps, box.r_cut)
    a = gt.force().double().cpu().numpy()
    rms, mx = rel_err(a, ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)
    idx = np.random.default_rng(1).choice(box.n, 2000, replace=False)
    brute = oracle.brute_force_sample(box.pos, box.mass, box.G, box.eps, box.r_cut, idx)
    assert rel_err(a[idx], brute)[0] <= TREE_RMS


@pytest.mark.slow
def test_clustered_2M_full_size():
    """The benchmark workload at full size: bit-exact keys and lists, FP32
    forces against the oracle's FP64 forces on identical lists."""
    box = inputs.config_box(2)
    gt = gpu_tree(box)
    ot = oracle_tree(box)
    assert_structure_equal(gt, ot)
    ref = ot.list_forces(box.G, box.eps, box.r_cut)
    rms, mx = rel_err(gt.force().double().cpu().numpy(), ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)
    assert gt.stats()["n_useful"] == ot.count_useful(box.eps, box.r_cut)


def test_vjp_against_oracle_adjoint():
    box = inputs.config_box(4, n_override=32768)
    w = inputs.cotangent(box.n, box.seed + 7)
    ot = oracle_tree(box)
    ref = ot.list_vjp(box.G, box.eps, box.r_cut, w.astype(np.float64))
    for prec in ["fp32", "fp64"]:
        gt = gpu_tree(box, prec)
        cot = torch.tensor(w, device="cuda")
        g = gt.vjp(cot).cpu().numpy()
        scale = max(np.sqrt(np.mean(ref ** 2)), 1e-300)
        tol = 1e-4 if prec == "fp32" else 1e-10
        bad = np.abs(g - ref) > tol * np.maximum(np.abs(ref), scale)
        assert not bad.any(), (prec, int(bad.sum()), float(np.abs(g - ref).max() / scale))


def test_batched_boxes_match_per_box_oracle():
    boxes = inputs.batched_boxes(8, scale=0.2)
    pos = torch.tensor(np.concatenate([b.pos for b in boxes]), device="cuda")
    mass = torch.tensor(np.concatenate([b.mass for b in boxes]), device="cuda")
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    prm = [Params(b.G, b.eps, b.r_cut, b.theta, b.n_crit, b.n_leaf, "fp32") for b in boxes]
    gt = ShortRangeTree(pos, mass, prm, box_offsets=offs.tolist())
    acc = gt.force().double().cpu().numpy()
    for k, b in enumerate(boxes):
        ref = oracle_tree(b).list_forces(b.G, b.eps, b.r_cut)
        rms, mx = rel_err(acc[offs[k]:offs[k + 1]], ref)
        assert rms <= FP32_RMS and mx <= FP32_MAX, (k, rms, mx)


def test_empty_and_errors():
    from paper_1211_4406_gb300._lib import TreeSRError
    t = ShortRangeTree(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), None, Params(r_cut=0.1))
    assert t.force().shape == (0, 3)
    assert t.stats()["n_groups"] == 0
    t.close()
    pos = torch.rand((100, 3), dtype=torch.float64, device="cuda")
    pos[17, 1] = float("nan")
    with pytest.raises(TreeSRError) as e:
        ShortRangeTree(pos, None, Params(r_cut=0.1))
    assert e.value.code == -6
    with pytest.raises(TreeSRError):
        ShortRangeTree(torch.rand((10, 3), dtype=torch.float64, device="cuda"), None, Params(r_cut=0.6))


def test_eps_zero_and_coincident_pairs_are_finite():
    pos = np.random.default_rng(3).random((2000, 3))
    pos[1000:1010] = pos[5]
    box = inputs.Box("eps0", pos, np.full(2000, 1 / 2000), 1.0, 0.0, 0.1, 0.5)
    a = gpu_tree(box).force().double().cpu().numpy()
    assert np.all(np.isfinite(a))
    ref = oracle_tree(box).list_forces(box.G, box.eps, box.r_cut)
    rms, mx = rel_err(a, ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX


def test_lognormal_masses_far_images_and_default_mass():
    """Masses spanning ~8 decades, G != 1, coordinates many boxes away from
    [0,1) (wrapped by both sides) and some exactly at 1.0: structure bit-exact,
    forces and the adjoint within the bounds; mass = None equals explicit 1/n."""
    rng = np.random.default_rng(4406)
    base = inputs.config_box(2, n_override=2 ** 15)
    mass = np.exp(rng.normal(0.0, 3.0, base.n)) / base.n
    shift = rng.integers(-5, 6, size=base.pos.shape).astype(np.float64)
    pos = base.pos + shift
    pos[:7, 0] = 1.0                              # the wrap of 1.0 is 0.0
    pos[7:11, 1] = -3.0
    box = inputs.Box("lognormal", pos, mass, 6.674e-3, base.eps, base.r_cut, base.theta)
    ot = oracle_tree(box)
    g32 = gpu_tree(box, "fp32")
    keys, perm = g32.export_keys()
    okeys = ot.export().keys
    assert np.array_equal(keys, okeys)
    ref = ot.list_forces(box.G, box.eps, box.r_cut)
    rms, mx = rel_err(g32.force().double().cpu().numpy(), ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)
    w = inputs.cotangent(box.n, 4407)
    gref = ot.list_vjp(box.G, box.eps, box.r_cut, w.astype(np.float64))
    scale = np.sqrt(np.mean(gref ** 2))
    g = g32.vjp(torch.tensor(w, device="cuda")).cpu().numpy()
    assert np.all(np.abs(g - gref) <= 1e-4 * np.maximum(np.abs(gref), scale))
    a2, g2 = g32.force_vjp(torch.tensor(w, device="cuda"))
    rms, mx = rel_err(a2.double().cpu().numpy(), ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)
    # the default mass (1/n) is the same as passing it
    p = torch.tensor(base.pos, device="cuda")
    prm = Params(base.G, base.eps, base.r_cut, base.theta, 64, 8, "fp32")
    t_none = ShortRangeTree(p, None, prm)
    t_expl = ShortRangeTree(p, torch.full((base.n,), 1.0 / base.n, dtype=torch.float64, device="cuda"), prm)
    assert torch.equal(t_none.force(), t_expl.force())


def test_rebuild_on_a_side_stream_and_from_a_graph_equals_a_fresh_build():
    """A build forks work onto the tree's own second stream and joins it back
    into the caller's stream: after a rebuild from new positions on another
    stream, and after a graph replay of the rebuild, the keys, nodes
    (monopoles included), groups, lists and one-pass forces equal those of a
    fresh build on the same positions."""
    pos0, mass = inputs.clustered_box(6000, 30, 77)
    pos1 = pos0 + 0.002 * np.sin(np.arange(pos0.size, dtype=np.float64).reshape(pos0.shape))
    prm = Params(1.3, 5e-4, 0.08, 0.5, 32, 4, "fp32")
    dev = torch.device("cuda")
    m = torch.tensor(mass, device=dev)
    cot = torch.tensor(inputs.cotangent(pos0.shape[0], 31), device=dev)
    fresh = ShortRangeTree(torch.tensor(pos1, device=dev), m, prm)
    ref = [fresh.export_keys(), fresh.export_nodes(), fresh.export_groups(), fresh.export_lists()]
    a_ref, _ = fresh.force_vjp(cot)
    a_ref = a_ref.clone()

    def same(t):
        got = [t.export_keys(), t.export_nodes(), t.export_groups(), t.export_lists()]
        for x, y in zip(got, ref):
            for u, v in zip(x, y):
                assert np.array_equal(u, v)

    t = ShortRangeTree(torch.tensor(pos0, device=dev), m, prm)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    t.rebuild(torch.tensor(pos1, device=dev), m, stream=side)
    assert t.status() == 0
    same(t)
    p = torch.tensor(pos0, device=dev)
    acc = torch.empty((t.n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((t.n, 3), dtype=torch.float64, device=dev)
    step = CapturedStep(t, p, m, cot, acc, grad)
    p.copy_(torch.tensor(pos1, device=dev))
    step.replay()
    torch.cuda.synchronize()
    assert t.status() == 0
    same(t)
    assert torch.equal(acc, a_ref)
    t.close()
    fresh.close()


@pytest.mark.parametrize("box", small_boxes() + [inputs.config_box(1), inputs.config_box(4)],
                         ids=lambda b: b.name)
def test_useful_pairs_bit_exact(box):
    """tp_stats.n_useful (evaluated pairs with a non-zero Eq. 2 term) equals
    the oracle's FP64 count on identical lists, for both cutoff arguments."""
    for xi in ("plain", "softened"):
        pos = torch.tensor(box.pos, device="cuda")
        mass = torch.tensor(box.mass, device="cuda")
        gt = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf,
                                              "fp32", xi=xi))
        st = gt.stats()
        gt.close()
        ot = oracle_tree(box)
        want = ot.count_useful(box.eps, box.r_cut, xi_softened=xi == "softened")
        assert st["n_useful"] == want, (xi, st["n_useful"], want)
        assert 0 <= st["n_useful"] <= st["n_interactions"]
