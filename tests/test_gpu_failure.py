"""Failure detection and determinism on the GPU, without faulting it.

- A walk that runs out of its node-visit budget ends its list and latches
  TP_ERR_TIMEOUT; the host reads it from tp_tree_status, the context stays
  usable, and a rebuild with the default budget gives the original forces.
  (The budget is the walk's only data-dependent loop bound; the library has
  no spin-waits on flags.)
- Rebuilding the same inputs reproduces keys, lists and FP32 forces bit for
  bit; the adjoint, summed with FP64 atomics, agrees to 1e-12 of its scale.
- A rebuild whose lists outgrow the capacities of the allocating build
  latches TP_ERR_LIST_OVERFLOW, and the forces and the adjoint of the
  following one-pass call are zeros (every kernel bounds its writes by the
  capacities and skips the lists once the status is latched).
"""
import numpy as np
import pytest
import torch

from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300._lib import TreeSRError
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu

TP_ERR_TIMEOUT = -5
TP_ERR_LIST_OVERFLOW = -4


def make_tree():
    box = inputs.config_box(2, n_override=2 ** 15)
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32")
    return box, pos, mass, ShortRangeTree(pos, mass, prm)


def test_walk_budget_exhaustion_is_reported_and_recoverable():
    box, pos, mass, t = make_tree()
    a0 = t.force().clone()
    t.set_walk_budget(3)
    t.rebuild(pos, mass)
    assert t.status() == TP_ERR_TIMEOUT
    with pytest.raises(TreeSRError):
        t.set_walk_budget(-1)
    t.set_walk_budget(0)
    t.rebuild(pos, mass)
    assert t.status() == 0
    assert torch.equal(t.force(), a0)
    t.close()


def test_rebuilds_are_deterministic():
    box, pos, mass, t1 = make_tree()
    _, _, _, t2 = make_tree()
    k1, p1 = t1.export_keys()
    k2, p2 = t2.export_keys()
    assert np.array_equal(k1, k2) and np.array_equal(p1, p2)
    o1, e1 = t1.export_lists()
    o2, e2 = t2.export_lists()
    assert np.array_equal(o1, o2) and np.array_equal(e1, e2)
    assert torch.equal(t1.force(), t2.force())
    cot = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device="cuda")
    g1, g2 = t1.vjp(cot), t2.vjp(cot)
    scale = float(g1.pow(2).mean().sqrt())
    assert float((g1 - g2).abs().max()) <= 1e-12 * scale
    a1, _ = t1.force_vjp(cot)
    t1.rebuild(pos, mass)
    a2, _ = t1.force_vjp(cot)
    assert torch.equal(a1, a2)
    t1.close()
    t2.close()


def test_rebuild_past_the_capacities_writes_zeros():
    n = 8192
    rng = np.random.default_rng(12)
    prm = Params(G=1.0, eps=1e-3, r_cut=0.05, theta=0.5, n_crit=64)
    t = ShortRangeTree(torch.tensor(rng.random((n, 3)), device="cuda"), None, prm)
    assert t.status() == 0
    # every particle within a 0.02 cube: each group's list holds all n
    # particles, far beyond the capacities taken from the uniform box
    t.rebuild(torch.tensor(0.5 + 0.02 * rng.random((n, 3)), device="cuda"), None)
    assert t.status() == TP_ERR_LIST_OVERFLOW
    cot = torch.tensor(inputs.cotangent(n, 13), device="cuda")
    acc = torch.full((n, 3), 7.0, dtype=torch.float32, device="cuda")
    grad = torch.full((n, 3), 7.0, dtype=torch.float64, device="cuda")
    t.force_vjp(cot, acc, grad)
    torch.cuda.synchronize()
    assert t.status() == TP_ERR_LIST_OVERFLOW
    assert not bool(acc.any()) and not bool(grad.any())
    t.close()
