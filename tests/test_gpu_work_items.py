"""Groups of more than 128 particles: the pair kernels take them as several
work items (chunks of 128 particles, each its own entry in the LPT order).
Forward, adjoint and the one pass, FP32 and FP64, packed and general
kernels, against the oracle on identical lists:

- a clustered box with n_crit = 320 (groups of up to 320 particles: three
  items), in the paper's kernel variants as well;
- a clump of 600 coincident particles (a leaf at the deepest level, so a
  group of 600 whatever n_crit: five items) in a uniform background;
- a tiny box whose groups span half of it (the general kernels, whose pair
  offsets take the minimum image per pair), and the clump with eps = 0 (also
  the general kernels).
Bounds as in test_gpu_parity.py (forces) and test_gpu_adjoint.py (adjoint),
except where the groups are wider than the workloads' (n_crit = 320 against
64): the FP32 rounding of the group-relative offsets grows with the width, so
the FP32 force rms is held to 2e-6 (measured 1.0e-6) and the FP32 adjoint, as
for the wide groups of the largest uniform C3 box, to at most 1e-4 of the
coordinates beyond 1e-4 and none beyond 1e-3 (measured max 2.9e-4: a close
pair amplified by the 1/s^5 term).  A chunk taken twice or missed would be an
O(1) error in many coordinates, and the FP64 path is held to 1e-8 (forces)
and 1e-10 (adjoint) throughout.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def coord_err(g, ref):
    scale = np.sqrt(np.mean(ref ** 2))
    return np.abs(g - ref) / np.maximum(np.abs(ref), scale)


def vjp_err(g, ref):
    return float(np.max(coord_err(g, ref)))


def boxes():
    pos, mass = inputs.clustered_box(32768, 20, 5)
    big = inputs.Box("clustered32k_ncrit320", pos, mass, 1.0, 1.0 / 3200, 3.0 / 32, 0.5, n_crit=320, n_leaf=8)
    rng = np.random.default_rng(9)
    bg = rng.random((20000, 3))
    clump = np.tile([[0.41, 0.52, 0.63]], (600, 1))
    pos = np.concatenate([bg, clump])
    mass = np.concatenate([np.full(20000, 1.0 / 20600), np.full(600, 0.5 / 20600)])
    coinc = inputs.Box("clump600", pos, mass, 1.0, 1.0 / 2000, 0.06, 0.5, n_crit=64, n_leaf=8)
    pos, mass = inputs.uniform_box(1500, 13)
    tiny = inputs.Box("tiny_box_spanning_groups", pos, mass, 1.0, 1e-3, 0.2, 0.5, n_crit=400, n_leaf=8)
    return [big, coinc, tiny]


def group_sizes(ot):
    return ot.export().gcount


@pytest.mark.parametrize("box", boxes(), ids=lambda b: b.name)
@pytest.mark.parametrize("variant", [{}, {"xi": "softened"}, {"rsqrt": "refined"}], ids=["plain", "xi_soft", "rsqrt"])
@pytest.mark.parametrize("adj_tile", [4, 8])
def test_large_groups_against_oracle(box, variant, adj_tile):
    soft = variant.get("xi") == "softened"
    refined = variant.get("rsqrt") == "refined"
    ot = oracle.OracleTree(box.pos, box.mass, box.n_leaf, box.n_crit)
    ot.lists(box.r_cut, box.theta)
    assert group_sizes(ot).max() > 256                     # at least three work items in one group
    w = inputs.cotangent(box.n, 21).astype(np.float64)
    ref = ot.list_forces(box.G, box.eps, box.r_cut, xi_softened=soft, rsqrt_refined=refined)
    gref = ot.list_vjp(box.G, box.eps, box.r_cut, w, xi_softened=soft, rsqrt_refined=refined)
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    cot = torch.tensor(w.astype(np.float32), device="cuda")
    for prec in ("fp64", "fp32"):
        if refined and prec == "fp64":
            continue                                        # the refined root is an FP32 variant
        t = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf,
                                             prec, **variant))
        t.set_tile(2, adj_tile)                             # 8: the entry-packed one pass
        c = cot if prec == "fp32" else cot.double()
        a = t.force().double().cpu().numpy()
        g = t.vjp(c).cpu().numpy()
        a1, g1 = t.force_vjp(c)
        a1, g1 = a1.double().cpu().numpy(), g1.cpu().numpy()
        t.close()
        rms, mx = rel_err(a, ref)
        if prec == "fp32":
            assert rms <= 2e-6 and mx <= 1e-4, (box.name, rms, mx)
            rms1, mx1 = rel_err(a1, ref)                    # the one pass sums in its own order
            assert rms1 <= 2e-6 and mx1 <= 1e-4, (box.name, rms1, mx1)
            for gg in (g, g1):
                e = coord_err(gg, gref)
                assert (e > 1e-4).mean() <= 1e-4 and e.max() <= 1e-3, (box.name, int((e > 1e-4).sum()), e.max())
        else:
            assert rms <= 1e-8, (box.name, rms)
            assert np.array_equal(a1, a)                    # FP64: the forward's forces bit for bit
            assert vjp_err(g, gref) <= 1e-10 and vjp_err(g1, gref) <= 1e-10


def test_large_groups_eps_zero_general_kernels():
    box = boxes()[1]               # the clump in a uniform background: no pair closer than the clump
    ot = oracle.OracleTree(box.pos, box.mass, box.n_leaf, box.n_crit)
    ot.lists(box.r_cut, box.theta)
    w = inputs.cotangent(box.n, 22).astype(np.float64)
    ref = ot.list_forces(box.G, 0.0, box.r_cut)
    gref = ot.list_vjp(box.G, 0.0, box.r_cut, w)
    t = ShortRangeTree(torch.tensor(box.pos, device="cuda"), torch.tensor(box.mass, device="cuda"),
                       Params(box.G, 0.0, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32"))
    a = t.force().double().cpu().numpy()
    g = t.vjp(torch.tensor(w.astype(np.float32), device="cuda")).cpu().numpy()
    t.close()
    rms, mx = rel_err(a, ref)
    assert rms <= 1e-6 and mx <= 1e-4, (rms, mx)
    assert vjp_err(g, gref) <= 1e-4
