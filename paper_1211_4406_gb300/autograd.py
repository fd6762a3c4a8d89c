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


# ---------------------------------------------------------------------------
# TreePM: the short-range force plus the long-range (PM) force, and the
# multiple-stepsize integrator of the paper's runs (one PM cycle and two PP
# cycles per step).
# ---------------------------------------------------------------------------
class PMForce(torch.autograd.Function):
    """a = PM(x): long-range accelerations (float32); backward = tp_pm_vjp."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, mass: torch.Tensor | None, pm):
        ctx.save_for_backward(pos)
        ctx.mass, ctx.pm = mass, pm
        return pm.force(pos.detach(), None if mass is None else mass.detach())

    @staticmethod
    def backward(ctx, g_acc: torch.Tensor):
        pos, = ctx.saved_tensors
        cot = g_acc.float().contiguous()
        return ctx.pm.vjp(pos.detach(), ctx.mass, cot), None, None


def pm_force(pos, mass, pm) -> torch.Tensor:
    return PMForce.apply(pos, mass, pm)


def _cot(like: torch.Tensor, dtype, *terms) -> torch.Tensor:
    """Sum of the (tensor or None, factor) terms in `dtype`, shaped like
    `like` (float64 accumulation in the library)."""
    acc = torch.zeros(like.shape, dtype=torch.float64, device=like.device)
    for t, f in terms:
        if t is not None:
            axpy(acc, t.contiguous(), f)
    if dtype == torch.float64:
        return acc
    out = torch.empty(acc.shape, dtype=dtype, device=acc.device)
    scale(out, acc, 1.0)
    return out


class TreePMStep(torch.autograd.Function):
    """(x, v, a_PP, a_PM) -> the same one multiple-stepsize step later:
        v += a_PM dt/2
        twice:  v += a_PP dt/4;  x += v dt/2;  a_PP = PP(x);  v += a_PP dt/4
        a_PM = PM(x);  v += a_PM dt/2
    With refit the second PP sub-step keeps the first one's tree structure and
    lists (tp_refit_tree) instead of rebuilding.  Only the inputs are saved
    (a checkpoint per step): backward recomputes the sub-step positions and
    their trees, then reverses each operation."""

    @staticmethod
    def forward(ctx, x, v, a_pp, a_pm, mass, params: Params, pm, dt: float, refit: bool, slots):
        h = 0.5 * dt
        vv = _copy64(v)
        axpy(vv, a_pm.contiguous(), 0.5 * dt)
        axpy(vv, a_pp.contiguous(), 0.5 * h)
        x1 = _copy64(x)
        axpy(x1, vv, h)
        t, a1 = _force(x1, mass, params, slots[0])
        axpy(vv, a1, h)                        # the first sub-step's closing kick and the second's opening one
        x2 = _copy64(x1)
        axpy(x2, vv, h)
        if refit:
            t.refit(x2, mass)
            a2 = t.force()
        else:
            t, a2 = _force(x2, mass, params, slots[0])
        axpy(vv, a2, 0.5 * h)
        am = pm.force(x2, mass)
        axpy(vv, am, 0.5 * dt)
        torch.cuda.current_stream().synchronize()
        ctx.save_for_backward(x, v, a_pp, a_pm)
        ctx.mass, ctx.params, ctx.pm, ctx.dt, ctx.refit, ctx.slots = mass, params, pm, dt, refit, slots
        return x2, vv, a2, am

    @staticmethod
    def backward(ctx, g_x2, g_v, g_app, g_apm):
        x, v, a_pp, a_pm = ctx.saved_tensors
        dt, h, mass, params, pm = ctx.dt, 0.5 * ctx.dt, ctx.mass, ctx.params, ctx.pm
        dev = x.device
        g_x2 = _zeros64(x.shape, dev) if g_x2 is None else g_x2
        g_v = _zeros64(x.shape, dev) if g_v is None else g_v
        # recompute the sub-step positions (and the first sub-step's force)
        vv = _copy64(v)
        axpy(vv, a_pm.contiguous(), 0.5 * dt)
        axpy(vv, a_pp.contiguous(), 0.5 * h)
        x1 = _copy64(x)
        axpy(x1, vv, h)
        s1, s2 = ctx.slots[1], ctx.slots[2]
        t1, a1 = _force(x1, mass, params, s1)
        axpy(vv, a1, h)
        x2 = _copy64(x1)
        axpy(x2, vv, h)
        # v += a_PM(x2) dt/2;  a_PM = PM(x2)
        gx = pm.vjp(x2, mass, _cot(x, torch.float32, (g_apm, 1.0), (g_v, 0.5 * dt)))
        axpy(gx, g_x2.contiguous(), 1.0)
        # v += a_PP(x2) dt/4;  a_PP = PP(x2)
        if ctx.refit:
            t1.refit(x2, mass)
            t2 = t1
        else:
            t2 = s2.tree_at(x2, mass, params)
            s2.check(x2, mass, params)
            t2 = s2.tree
        axpy(gx, t2.vjp(_cot(x, t2.acc_dtype, (g_app, 1.0), (g_v, 0.5 * h))), 1.0)
        gv = _copy64(g_v)
        axpy(gv, gx, h)                                  # x2 = x1 + v h
        if ctx.refit:
            t1.refit(x1, mass)                           # back to the build positions
        # v += a_PP(x1) dt/4 twice;  a_PP = PP(x1)
        axpy(gx, t1.vjp(_cot(x, t1.acc_dtype, (gv, h))), 1.0)
        axpy(gv, gx, h)                                  # x1 = x + v h
        g_a_pp = torch.empty(x.shape, dtype=a_pp.dtype, device=dev)
        scale(g_a_pp, gv, 0.5 * h)
        g_a_pm = torch.empty(x.shape, dtype=a_pm.dtype, device=dev)
        scale(g_a_pm, gv, 0.5 * dt)
        torch.cuda.current_stream().synchronize()
        return gx, gv, g_a_pp, g_a_pm, None, None, None, None, None, None


def treepm_leapfrog(x0: torch.Tensor, v0: torch.Tensor, mass, params: Params, pm, dt: float, steps: int,
                    refit: bool = False):
    """Integrate `steps` multiple-stepsize TreePM steps (PM solver `pm` with
    the same r_cut and G as params); returns (x_T, v_T, a_PP(x_T), a_PM(x_T)).
    Differentiable in x0 and v0 with one checkpoint per step.  The steps share
    one tree for the forward pass and two for the backward pass, rebuilt in
    place.  refit needs whole lists (a tree in chunked mode refuses it)."""
    a_pp = short_range_force(x0, mass, params)
    a_pm = pm_force(x0, mass, pm)
    slots = (_TreeSlot(), _TreeSlot(), _TreeSlot())
    x, v = x0, v0
    for _ in range(steps):
        x, v, a_pp, a_pm = TreePMStep.apply(x, v, a_pp, a_pm, mass, params, pm, dt, refit, slots)
    return x, v, a_pp, a_pm
