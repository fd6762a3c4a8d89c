"""Differentiable short-range force and a checkpointed kick-drift-kick leapfrog.

ShortRangeForce: forward = tree build + Eq. 2 on the lists (tp_build_tree +
tp_short_range_force); backward = tp_short_range_vjp on the same tree (walk
decisions are piecewise constant and not differentiated).

KDKStep: one leapfrog step with the short-range force only (the steps of one
chain reuse a forward tree and a backward tree, rebuilt in place),
    v_h = v + a dt/2,  x1 = x + v_h dt,  a1 = F(x1),  v1 = v_h + a1 dt/2,
saving only its inputs (x, v, a): backward rebuilds the tree at x1 (the
recomputation that makes every step a checkpoint) and chains the adjoint
    g_a1' = g_a1 + (dt/2) g_v1
    g_x1' = g_x1 + VJP_F(x1)[g_a1']
    g_vh  = g_v1 + dt g_x1'
    g_x = g_x1',  g_v = g_vh,  g_a = (dt/2) g_vh.
Every update, copy and cast runs in the library (tp_axpy / tp_scale); torch
only allocates.
"""
from __future__ import annotations

import torch

from .api import Params, ShortRangeTree, axpy, scale


def _copy64(x: torch.Tensor) -> torch.Tensor:
    """FP64 copy of x (float32 or float64), made by a library kernel."""
    if x.dtype == torch.float64:
        out = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        scale(out, x.contiguous(), 1.0)
    else:
        out = torch.zeros(x.shape, dtype=torch.float64, device=x.device)
        axpy(out, x.contiguous(), 1.0)
    return out


def _zeros64(shape, device) -> torch.Tensor:
    return torch.zeros(shape, dtype=torch.float64, device=device)


class ShortRangeForce(torch.autograd.Function):
    """a = F(x): short-range accelerations of Eq. 2 (dtype of the precision)."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, mass: torch.Tensor | None, params: Params):
        tree = ShortRangeTree(pos.detach(), None if mass is None else mass.detach(), params)
        acc = tree.force()
        ctx.tree = tree
        return acc

    @staticmethod
    def backward(ctx, g_acc: torch.Tensor):
        tree = ctx.tree
        grad = tree.vjp(g_acc.contiguous())
        tree.close()
        ctx.tree = None
        return grad, None, None


def short_range_force(pos, mass, params: Params) -> torch.Tensor:
    return ShortRangeForce.apply(pos, mass, params)


class _TreeSlot:
    """One tree reused across the steps of a leapfrog chain: rebuilt in place
    (no allocation) from each step's positions, replaced by a fresh allocating
    build when a rebuild exceeded the capacities of the tree's first build
    (the step synchronises anyway, so the latched status is read there)."""

    def __init__(self):
        self.tree = None

    def tree_at(self, x, mass, params):
        if self.tree is None:
            self.tree = ShortRangeTree(x, mass, params)
        else:
            self.tree.rebuild(x, mass)
        return self.tree

    def check(self, x, mass, params) -> bool:
        """True if the last rebuild was good; else rebuilds with allocation."""
        if self.tree.status() == 0:
            return True
        self.tree.close()
        self.tree = ShortRangeTree(x, mass, params)
        return False

    def close(self):
        if self.tree is not None:
            self.tree.close()
            self.tree = None


def _force(x, mass, params, slot: _TreeSlot | None = None):
    if slot is None:
        t = ShortRangeTree(x, mass, params)
        return t, t.force()
    t = slot.tree_at(x, mass, params)
    a = t.force()
    if not slot.check(x, mass, params):
        a = slot.tree.force()
    return slot.tree, a


class KDKStep(torch.autograd.Function):
    """(x, v, a) -> (x1, v1, a1), one checkpointed kick-drift-kick step."""

    @staticmethod
    def forward(ctx, x, v, a, mass, params: Params, dt: float, slots=None):
        vh = _copy64(v)
        axpy(vh, a.contiguous(), 0.5 * dt)
        x1 = _copy64(x)
        axpy(x1, vh, dt)
        t, a1 = _force(x1, mass, params, None if slots is None else slots[0])
        v1 = _copy64(vh)
        axpy(v1, a1, 0.5 * dt)
        torch.cuda.current_stream().synchronize()
        if slots is None:
            t.close()
        ctx.save_for_backward(x, v, a)
        ctx.mass, ctx.params, ctx.dt, ctx.slots = mass, params, dt, slots
        ctx.a_dtype = a.dtype
        return x1, v1, a1

    @staticmethod
    def backward(ctx, g_x1, g_v1, g_a1):
        x, v, a = ctx.saved_tensors
        dt = ctx.dt
        dev = x.device
        g_x1 = _zeros64(x.shape, dev) if g_x1 is None else g_x1
        g_v1 = _zeros64(x.shape, dev) if g_v1 is None else g_v1
        # recompute the step's position and rebuild its tree (checkpoint)
        vh = _copy64(v)
        axpy(vh, a.contiguous(), 0.5 * dt)
        x1 = _copy64(x)
        axpy(x1, vh, dt)
        slot = None if ctx.slots is None else ctx.slots[1]
        if slot is None:
            tree = ShortRangeTree(x1, ctx.mass, ctx.params)
        else:
            slot.tree_at(x1, ctx.mass, ctx.params)
            slot.check(x1, ctx.mass, ctx.params)
            tree = slot.tree
        # g_a1' = g_a1 + (dt/2) g_v1, in the force's precision
        ga = torch.empty(x.shape, dtype=torch.float64, device=dev)
        scale(ga, g_v1.contiguous(), 0.5 * dt)
        if g_a1 is not None:
            axpy(ga, g_a1.contiguous(), 1.0)
        cot = torch.empty(x.shape, dtype=tree.acc_dtype, device=dev)
        scale(cot, ga, 1.0)
        gx = tree.vjp(cot)                               # VJP_F(x1)[g_a1']
        axpy(gx, g_x1.contiguous(), 1.0)                 # g_x1' = g_x1 + ...
        gvh = _copy64(g_v1)
        axpy(gvh, gx, dt)                                # g_vh = g_v1 + dt g_x1'
        g_a = torch.empty(x.shape, dtype=ctx.a_dtype, device=dev)
        scale(g_a, gvh, 0.5 * dt)                        # g_a = (dt/2) g_vh
        torch.cuda.current_stream().synchronize()
        if slot is None:
            tree.close()
        return gx, gvh, g_a, None, None, None, None


def leapfrog(x0: torch.Tensor, v0: torch.Tensor, mass, params: Params, dt: float, steps: int,
             reuse_trees: bool = True):
    """Integrate `steps` KDK steps from (x0, v0); returns (x_T, v_T, a_T).
    Differentiable in x0 and v0 with one checkpoint (x, v, a) per step.  With
    reuse_trees the steps share one tree for the forward pass and one for the
    backward pass, rebuilt in place (the trees are freed with the graph)."""
    a = short_range_force(x0, mass, params)
    slots = (_TreeSlot(), _TreeSlot()) if reuse_trees else None
    x, v = x0, v0
    for _ in range(steps):
        x, v, a = KDKStep.apply(x, v, a, mass, params, dt, slots)
    return x, v, a
