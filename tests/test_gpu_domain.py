"""The device side of the spatial decomposition (csrc/tp_domain.cu through the
C-ABI): owner and ghost selections bit-exact against the oracle (indices,
order and counts), the row gather and scatter-add, and one step of an
8-domain decomposition emulated on one GPU -- every domain's own particles
followed by the ghosts the other domains select for it, a tree over them,
forces and adjoint in one pass, ghost gradients added back to their owners --
against the oracle's single-box direct sum and adjoint (theta = 0) and within
the tree's accuracy (theta = 0.5).  The collectives between ranks are covered
by tests/test_domain_host.py (gloo on CPU); DomainShortRange is run here as
one rank."""
import numpy as np
import pytest
import torch

import oracle
from oracle import domain as od
from paper_1211_4406_gb300 import domain as dom
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300._lib import TreeSRError
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu


def geometry(seed, shape):
    rng = np.random.default_rng(seed)
    pos, _ = inputs.clustered_box(20000, 20, seed)
    g = dom.multisection(pos[rng.choice(pos.shape[0], 4000, replace=False)], *shape)
    return g


def test_selections_match_the_oracle_bit_for_bit():
    g = geometry(7, (3, 2, 2))
    pos, _ = inputs.clustered_box(50000, 30, 8)
    pos[:4] = [[g.xc[1], g.yc[0, 1], g.zc[0, 0, 1]], [1.0, 0.0, -0.0], [-3.0, 2.5, 7.25], [0.5, 1.0 - 1e-17, 0.2]]
    pos[4:20] += np.random.default_rng(1).integers(-3, 4, (16, 3))
    halo = dom.Halo(*g.shape)
    halo.set_geometry(g)
    dp = torch.tensor(pos, device="cuda")
    idx, counts = halo.select(dp, "owner")
    oi, oc = od.select(pos, g.xc, g.yc, g.zc, "owner")
    assert counts == oc.tolist() and np.array_equal(idx.cpu().numpy(), oi)
    for self_d in (0, 5, 11):
        for rc in (0.03, 0.11):
            idx, counts = halo.select(dp, "ghosts", self_d, rc)
            oi, oc = od.select(pos, g.xc, g.yc, g.zc, "ghosts", self_d, rc)
            assert counts == oc.tolist() and np.array_equal(idx.cpu().numpy(), oi), (self_d, rc)
    bad = dp.clone()
    bad[3, 2] = float("nan")
    with pytest.raises(TreeSRError) as e:
        halo.select(bad, "owner")
    assert e.value.code == -6
    with pytest.raises(TreeSRError):
        halo.set_geometry(dom.Geometry(np.array([0.0, 0.7, 0.6, 1.0]), g.yc, g.zc))    # cuts out of order
    halo.close()


def test_gather_and_scatter_rows():
    torch.manual_seed(2)
    src = torch.randn((1000, 3), dtype=torch.float64, device="cuda")
    ids = torch.arange(1000, dtype=torch.int64, device="cuda") * 7
    f32 = torch.randn((1000, 3), dtype=torch.float32, device="cuda")
    idx = torch.randint(0, 1000, (3000,), dtype=torch.int32, device="cuda")
    assert torch.equal(dom.gather_rows(src, idx), src[idx.long()])
    assert torch.equal(dom.gather_rows(ids, idx), ids[idx.long()])
    assert torch.equal(dom.gather_rows(f32, idx), f32[idx.long()])
    assert torch.equal(dom.gather_rows(src[:, 0].contiguous(), idx), src[idx.long(), 0])
    dst = torch.zeros((1000, 3), dtype=torch.float64, device="cuda")
    vals = torch.randn((3000, 3), dtype=torch.float64, device="cuda")
    dom.scatter_add_rows(dst, idx, vals)
    want = torch.zeros_like(dst).index_add_(0, idx.long(), vals)
    assert float((dst - want).abs().max()) <= 1e-12


def emulated_step(pos, mass, w, g, prm):
    """One step of the decomposition with every domain on this GPU in turn:
    the data each rank would send and receive, without a collective."""
    n, nd = pos.shape[0], g.ndom
    halo = dom.Halo(*g.shape)
    halo.set_geometry(g)
    dp, dm = torch.tensor(pos, device="cuda"), torch.tensor(mass, device="cuda")
    dw = torch.tensor(w, device="cuda")
    oidx, oc = halo.select(dp, "owner")
    off = np.concatenate([[0], np.cumsum(oc)])
    own = [oidx[off[d]:off[d + 1]].long() for d in range(nd)]
    # ghosts: domain e's particles selected for domain d
    sent = {}
    for e in range(nd):
        gidx, gc = halo.select(dp[own[e]].contiguous(), "ghosts", e, prm.r_cut)
        goff = np.concatenate([[0], np.cumsum(gc)])
        for d in range(nd):
            sent[(e, d)] = own[e][gidx[goff[d]:goff[d + 1]].long()]
    acc = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    grad = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    nghost = 0
    for d in range(nd):
        gl = torch.cat([sent[(e, d)] for e in range(nd) if e != d])
        nghost += gl.numel()
        rows = torch.cat([own[d], gl])
        tree = ShortRangeTree(dp[rows].contiguous(), dm[rows].contiguous(), prm)
        cot = torch.cat([dw[own[d]], torch.zeros((gl.numel(), 3), dtype=torch.float32, device="cuda")])
        a, gr = tree.force_vjp(cot)
        tree.close()
        nl = own[d].numel()
        acc[own[d]] = a[:nl]
        dom.scatter_add_rows(grad, rows.int(), gr)            # own rows and the ghosts' share, to the owners
    halo.close()
    return acc.double().cpu().numpy(), grad.cpu().numpy(), nghost


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def test_emulated_eight_domain_step_matches_the_single_box():
    box = inputs.config_box(4, n_override=32768)
    w = inputs.cotangent(box.n, box.seed + 7)
    g = geometry(11, (2, 2, 2))
    ref = oracle.brute_force(box.pos, box.mass, box.G, box.eps, box.r_cut)
    gref = oracle.brute_vjp(box.pos, box.mass, box.G, box.eps, box.r_cut, w.astype(np.float64))
    for theta in (0.0, 0.5):
        prm = Params(box.G, box.eps, box.r_cut, theta, box.n_crit, box.n_leaf, "fp32")
        acc, grad, nghost = emulated_step(box.pos, box.mass, w, g, prm)
        assert nghost > 0
        rms, mx = rel_err(acc, ref)
        if theta == 0.0:
            assert rms <= 1e-6 and mx <= 1e-4, (rms, mx)
            scale = np.sqrt(np.mean(gref ** 2))
            bad = np.abs(grad - gref) > 1e-4 * np.maximum(np.abs(gref), scale)
            assert not bad.any(), (int(bad.sum()), float(np.abs(grad - gref).max() / scale))
        else:
            assert rms <= 5e-3, rms


def test_one_rank_step_equals_the_tree():
    box = inputs.config_box(4, n_override=8192)
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32")
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    cot = torch.tensor(inputs.cotangent(box.n, 3), device="cuda")
    ds = dom.DomainShortRange(prm)
    ds.update_geometry(pos, 1.0)
    p, m, ids = ds.exchange(pos, mass, torch.arange(box.n, dtype=torch.int64, device="cuda"))
    assert torch.equal(ids, torch.arange(box.n, dtype=torch.int64, device="cuda"))
    a, gr = ds.step(p, m, cot)
    t = ShortRangeTree(pos, mass, prm)
    a0, g0 = t.force_vjp(cot)
    t.close()
    assert torch.equal(a, a0)
    assert float((gr - g0).abs().max()) <= 1e-12 * float(g0.abs().max())
