"""tp_refit_tree: the structure, groups and lists of the last build are kept;
positions, monopoles and entry records are refreshed.  Checked against the
oracle's frozen-structure refresh (the same reading: each particle at the
image nearest its build position, node sums in the build's canonical order):
node masses and centres of mass bit for bit, forces and the adjoint within
the FP32 bounds -- with particles that cross the box boundary, a second refit
taken relative to the build, and a rebuild that moves the reference."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300._lib import TreeSRError
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def moved(pos, seed, amp):
    rng = np.random.default_rng(seed)
    p = pos + amp * rng.normal(size=pos.shape)
    edge = np.where(pos[:, 0] < 2 * amp)[0][:20]     # push a few across x = 0
    p[edge, 0] -= 4 * amp
    return p


def check(gt, ot, box, w):
    ints, dbl = gt.export_nodes()
    ex = ot.export()
    assert np.array_equal(dbl[:, 0], ex.M) and np.array_equal(dbl[:, 1:4], ex.com)
    rms, mx = rel_err(gt.force().double().cpu().numpy(), ot.list_forces(box.G, box.eps, box.r_cut))
    assert rms <= 1e-6 and mx <= 1e-4, (rms, mx)
    gref = ot.list_vjp(box.G, box.eps, box.r_cut, w.astype(np.float64))
    scale = np.sqrt(np.mean(gref ** 2))
    g = gt.vjp(torch.tensor(w, device="cuda")).cpu().numpy()
    assert np.all(np.abs(g - gref) <= 1e-4 * np.maximum(np.abs(gref), scale))


def test_refit_matches_oracle_refresh():
    box = inputs.config_box(2, n_override=2 ** 15)
    w = inputs.cotangent(box.n, box.seed + 7)
    amp = 1e-3 * box.r_cut
    prm = Params(box.G, box.eps, box.r_cut, box.theta, 64, 8, "fp32")
    gt = ShortRangeTree(torch.tensor(box.pos, device="cuda"), torch.tensor(box.mass, device="cuda"), prm)
    ot = oracle.OracleTree(box.pos, box.mass, 8, 64)
    ot.lists(box.r_cut, box.theta)
    p1 = moved(box.pos, 1, amp)
    assert (p1[:, 0] < 0).any()                      # some particles crossed the boundary
    gt.refit(torch.tensor(p1, device="cuda"))
    ot.refresh(p1)
    check(gt, ot, box, w)
    p2 = moved(box.pos, 2, amp)                      # relative to the build, not to p1
    gt.refit(torch.tensor(p2, device="cuda"))
    ot.refresh(p2)
    check(gt, ot, box, w)
    # a rebuild moves the reference
    gt.rebuild(torch.tensor(p2, device="cuda"))
    ot2 = oracle.OracleTree(p2, box.mass, 8, 64)
    ot2.lists(box.r_cut, box.theta)
    p3 = moved(p2, 3, amp)
    gt.refit(torch.tensor(p3, device="cuda"))
    ot2.refresh(p3)
    check(gt, ot2, box, w)
    assert gt.status() == 0
    gt.close()


def test_refit_refused_in_chunked_mode():
    box = inputs.config_box(2, n_override=2 ** 14)
    pos = torch.tensor(box.pos, device="cuda")
    t = ShortRangeTree(pos, None, Params(box.G, box.eps, box.r_cut, box.theta, 64, 8, "fp32", chunked=True))
    with pytest.raises(TreeSRError):
        t.refit(pos)
    t.close()
