"""GPU parity of the multiple-stepsize TreePM integrator (one PM cycle and
two PP cycles per step, the paper's schedule) and of its gradient, against
the oracle's integration and adjoint, with the second PP sub-step rebuilt or
refitted.

Bounds: the displacement x_T - x_0 and the velocity change within 1e-4 of
max(|ref|, rms(ref)) per coordinate (FP32 forces, ~1e-6 relative, over three
steps); the gradient in x_0 and v_0 of L = w_x.x_T + w_v.v_T + w_a.a_PP(x_T)
+ w_m.a_PM(x_T) within 1e-4 of max(|ref|, rms(ref)), the bound of the
short-range adjoint.
"""
import numpy as np
import pytest
import torch

from oracle import pm as opm
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300.api import Params, PMSolver
from paper_1211_4406_gb300.autograd import treepm_leapfrog

pytestmark = pytest.mark.gpu


def close(a, ref, tol):
    scale = np.sqrt(np.mean(ref ** 2))
    bad = np.abs(a - ref) > tol * np.maximum(np.abs(ref), scale)
    return not bad.any(), int(bad.sum()), float(np.abs(a - ref).max() / scale)


@pytest.mark.parametrize("refit", [False, True])
def test_treepm_leapfrog_and_gradient_match_oracle(refit):
    n = 4096
    pos, mass = inputs.clustered_box(n, 12, 71)
    rng = np.random.default_rng(72)
    vel = 0.05 * rng.normal(size=pos.shape)
    G, eps, n_mesh, theta, dt, steps = 1.0, 1e-2, 16, 0.5, 2e-4, 3
    rc = 3.0 / n_mesh
    xT, vT, aT, mT, evals = opm.treepm_leapfrog(pos, vel, mass, G, eps, rc, theta, n_mesh, dt, steps,
                                                n_crit=32, refit=refit)
    w = [rng.normal(size=pos.shape) for _ in range(4)]
    gx_ref, gv_ref = opm.treepm_leapfrog_adjoint(pos, vel, mass, evals, G, eps, rc, n_mesh, dt, steps, *w)

    dev = torch.device("cuda")
    x0 = torch.tensor(pos, device=dev, requires_grad=True)
    v0 = torch.tensor(vel, device=dev, requires_grad=True)
    m = torch.tensor(mass, device=dev)
    pm = PMSolver(n_mesh, rc, G)
    prm = Params(G, eps, rc, theta, 32, 8, "fp32")
    x, v, a, am = treepm_leapfrog(x0, v0, m, prm, pm, dt, steps, refit=refit)
    wt = [torch.tensor(t, device=dev) for t in w]
    loss = (wt[0] * x).sum() + (wt[1] * v).sum() + (wt[2] * a.double()).sum() + (wt[3] * am.double()).sum()
    loss.backward()

    ok = close(x.detach().cpu().numpy() - pos, xT - pos, 1e-4)
    assert ok[0], ("x", ok)
    ok = close(v.detach().cpu().numpy() - vel, vT - vel, 1e-4)
    assert ok[0], ("v", ok)
    ok = close(x0.grad.cpu().numpy(), gx_ref, 1e-4)
    assert ok[0], ("dL/dx0", ok)
    ok = close(v0.grad.cpu().numpy(), gv_ref, 1e-4)
    assert ok[0], ("dL/dv0", ok)
    pm.close()
