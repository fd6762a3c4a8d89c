"""The adjoint workload at its full size and coordinate count: N = 64^3 =
262,144 clustered particles (250 NFW halos, r_cut = 3/64, eps = 1/3200),
cotangent w ~ N(0,1), 64 seeded coordinates.  Minutes of CPU oracle work, so
these run only with TP_ONEOFF=1 (the default GPU suite checks the same things
on the N = 8192 and 32768 cuts of the recipe).

1. One force evaluation: the GPU VJP, FP32 and FP64, against FP64 Richardson
   central differences (h = 1e-4 eps and h/2) of the oracle's frozen-structure
   forces: |g - g_fd| <= 1e-4 max(|g_fd|, rms(g_ref)).
2. Ten KDK steps (dt = 1e-3): the GPU FP64 gradient against the oracle's
   analytic adjoint of the same trajectory on all 3N coordinates (1e-8), the
   FP32 gradient against it: median <= 1e-6 per coordinate and rms <= 1e-2.
   The clustered box amplifies any perturbation of the state over 10 steps,
   and more so at larger N (more close pairs): the FP32 chain measured rms
   5.7e-4 at N = 32768 and 3.8e-3 at N = 262144 (median 1.3e-9), the error
   sitting on the few coordinates in close encounters.  The test also prints
   how far the FP64 chain's own gradient moves when x0 is merely rounded to
   FP32, the size of perturbation the FP32 path makes at every step.
3. Ten KDK steps, FP64, on the N = 32768 cut of the recipe: the GPU gradient
   against Richardson differences of the oracle's frozen 10-step chain on 64
   coordinates."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300.api import Params
from paper_1211_4406_gb300.autograd import leapfrog, short_range_force

pytestmark = [pytest.mark.gpu, pytest.mark.oneoff]
TOL = 1e-4


def richardson(f, h):
    d = lambda s: (f(s) - f(-s)) / (2 * s)
    return (4 * d(h / 2) - d(h)) / 3


def coords_of(n, seed, count=64):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(n)), int(rng.integers(3))) for _ in range(count)]


def gpu_vjp(box, w, precision):
    pos = torch.tensor(box.pos, device="cuda", requires_grad=True)
    mass = torch.tensor(box.mass, device="cuda")
    acc = short_range_force(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, 64, 8, precision))
    (acc.double() * torch.tensor(w, device="cuda", dtype=torch.float64)).sum().backward()
    return pos.grad.cpu().numpy()


def test_c4_vjp_against_frozen_differences_64_coordinates():
    box = inputs.config_box(4)
    assert box.n == 64 ** 3
    w = inputs.cotangent(box.n, box.seed + 7).astype(np.float64)
    ot = oracle.OracleTree(box.pos, box.mass, 8, 64)
    ot.lists(box.r_cut, box.theta)
    ref = ot.list_vjp(box.G, box.eps, box.r_cut, w)
    scale = np.sqrt(np.mean(ref ** 2))
    coords = coords_of(box.n, 4406)
    fd = []
    for k, c in coords:
        def f(s):
            p = box.pos.copy()
            p[k, c] += s
            ot.refresh(p)
            return np.sum(w * ot.list_forces(box.G, box.eps, box.r_cut))
        fd.append(richardson(f, 1e-4 * box.eps))
    ot.refresh(box.pos)
    fd = np.array(fd)
    worst = {}
    for prec in ("fp32", "fp64"):
        g = gpu_vjp(box, w.astype(np.float32), prec)
        gk = np.array([g[k, c] for k, c in coords])
        e = np.abs(gk - fd) / np.maximum(np.abs(fd), scale)
        worst[prec] = float(e.max())
        assert e.max() <= TOL, (prec, float(e.max()))
        # and the whole gradient against the oracle's analytic VJP on the same lists
        eg = np.abs(g - ref) / np.maximum(np.abs(ref), scale)
        assert eg.max() <= (TOL if prec == "fp32" else 1e-8), (prec, float(eg.max()))
    print("C4 VJP vs FD, worst relative error over 64 coordinates:", worst)


def run_leapfrog(box, w, precision, steps, dt):
    x0 = torch.tensor(box.pos, device="cuda", requires_grad=True)
    v0 = torch.zeros_like(x0)
    mass = torch.tensor(box.mass, device="cuda")
    _, _, aT = leapfrog(x0, v0, mass, Params(box.G, box.eps, box.r_cut, box.theta, 64, 8, precision),
                        dt, steps)
    (aT.double() * torch.tensor(w, device="cuda", dtype=torch.float64)).sum().backward()
    return x0.grad.cpu().numpy()


def test_c4_ten_step_leapfrog_against_oracle_adjoint():
    box = inputs.config_box(4)
    w = inputs.cotangent(box.n, box.seed + 7).astype(np.float64)
    steps, dt = 10, 1e-3
    v0 = np.zeros_like(box.pos)
    _, _, _, trees = oracle.leapfrog(box.pos, v0, box.mass, box.G, box.eps, box.r_cut, box.theta,
                                     dt, steps, keep_trees=True)
    gref, _ = oracle.leapfrog_adjoint(box.pos, v0, trees, box.G, box.eps, box.r_cut, dt, steps,
                                      np.zeros_like(v0), np.zeros_like(v0), w)
    scale = np.sqrt(np.mean(gref ** 2))
    g64 = run_leapfrog(box, w, "fp64", steps, dt)
    e64 = np.abs(g64 - gref) / np.maximum(np.abs(gref), scale)
    assert e64.max() <= 1e-8, float(e64.max())
    g32 = run_leapfrog(box, w, "fp32", steps, dt)
    e32 = np.abs(g32 - gref) / np.maximum(np.abs(gref), scale)
    rms32 = float(np.sqrt(np.mean((g32 - gref) ** 2)) / scale)
    # sensitivity: the FP64 chain started from x0 rounded to FP32
    rounded = inputs.Box(box.name, box.pos.astype(np.float32).astype(np.float64), box.mass, box.G, box.eps,
                         box.r_cut, box.theta, seed=box.seed)
    g64r = run_leapfrog(rounded, w, "fp64", steps, dt)
    sens = float(np.sqrt(np.mean((g64r - g64) ** 2)) / scale)
    print("C4 10-step gradient: FP64 max", float(e64.max()), "FP32 rms", rms32, "median",
          float(np.median(e32)), "FP64 chain from FP32-rounded x0: rms change", sens)
    assert np.median(e32) <= 1e-6 and rms32 <= 1e-2, (rms32, float(np.median(e32)))


def test_c4_recipe_ten_step_leapfrog_against_frozen_differences_64_coordinates():
    box = inputs.config_box(4, n_override=2 ** 15)
    w = inputs.cotangent(box.n, box.seed + 7).astype(np.float64)
    steps, dt = 10, 1e-3
    v0 = np.zeros_like(box.pos)
    _, _, _, trees = oracle.leapfrog(box.pos, v0, box.mass, box.G, box.eps, box.r_cut, box.theta,
                                     dt, steps, keep_trees=True)
    gref, _ = oracle.leapfrog_adjoint(box.pos, v0, trees, box.G, box.eps, box.r_cut, dt, steps,
                                      np.zeros_like(v0), np.zeros_like(v0), w)
    scale = np.sqrt(np.mean(gref ** 2))
    g = run_leapfrog(box, w, "fp64", steps, dt)
    worst = 0.0
    for k, c in coords_of(box.n, 4407):
        def f(s):
            p = box.pos.copy()
            p[k, c] += s
            return np.sum(w * oracle.leapfrog_frozen(p, v0, trees, box.G, box.eps, box.r_cut, dt, steps)[2])
        fd = richardson(f, 1e-4 * box.eps)
        e = abs(g[k, c] - fd) / max(abs(fd), scale)
        worst = max(worst, e)
        assert e <= TOL, (k, c, g[k, c], fd)
    print("C4-recipe (N=32768) 10-step FP64 gradient vs FD, worst over 64 coordinates:", worst)
