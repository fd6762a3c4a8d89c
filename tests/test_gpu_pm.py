"""GPU parity of the long-range (PM) half against the PM oracle (Sec. II's PM
cycle), through the C-ABI.

The GPU mesh, FFTs and interpolation are FP32, the oracle FP64.  Bounds,
relative to the rms of the reference: potential and mesh acceleration rms
<= 1e-5; particle accelerations rms <= 1e-5 and max <= 1e-3 (with the same
1e-6 x median guard as the short-range tests).  Full-size case: the
clustered 2M box on its 128^3 mesh (r_cut = 3/128, three mesh spacings).
The PM + PP total through the library meets the oracle's Ewald bound.
"""
import numpy as np
import pytest
import torch

import oracle
from ewald_ref import ewald
from oracle import pm as opm
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300._lib import TreeSRError
from paper_1211_4406_gb300.api import Params, PMSolver, ShortRangeTree

pytestmark = pytest.mark.gpu


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def mesh_rel(a, ref):
    return float(np.sqrt(np.mean((a - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


def cases():
    rng = np.random.default_rng(11)
    out = []
    pos = rng.random((500, 3))
    pos[:5] += np.array([3.0, -2.0, 7.0])          # far images
    pos[5] = [1.0, 0.0, 0.999999999]               # exactly on the boundary
    out.append(("random500-mesh16", pos, rng.random(500) + 0.5, 16, 1.3))
    box = inputs.config_box(1)                     # uniform 32^3
    out.append(("uniform32k-mesh32", box.pos, None, 32, 1.0))
    box = inputs.config_box(2, n_override=2 ** 15)
    out.append(("clustered32k-mesh32", box.pos, box.mass * np.linspace(0.5, 1.5, box.n), 32, 1.0))
    box = inputs.config_box(2, n_override=2 ** 15)
    out.append(("clustered32k-mesh24", box.pos, None, 24, 0.7))
    return out


@pytest.mark.parametrize("name,pos,mass,n_mesh,G", cases(), ids=[c[0] for c in cases()])
def test_pm_matches_oracle(name, pos, mass, n_mesh, G):
    rc = 3.0 / n_mesh
    n = pos.shape[0]
    m_ref = np.full(n, 1.0 / n) if mass is None else mass
    rho = opm.assign(pos, m_ref, n_mesh)
    phi = opm.potential(rho, opm.green(n_mesh, rc, G))
    amesh = opm.gradient(phi)
    ref = opm.interpolate(pos, amesh)
    solver = PMSolver(n_mesh, rc, G)
    p = torch.tensor(pos, device="cuda")
    m = None if mass is None else torch.tensor(mass, device="cuda")
    acc = solver.force(p, m).double().cpu().numpy()
    assert mesh_rel(solver.export_mesh("potential"), phi) <= 1e-5
    assert mesh_rel(solver.export_mesh("acceleration"), np.stack(amesh, axis=-1)) <= 1e-5
    rms, mx = rel_err(acc, ref)
    assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
    # accumulate adds onto what is there; the two calls' FP32 atomic adds into
    # the mass mesh land in different orders (measured up to 1.3e-6 of max|a|)
    base = torch.full((n, 3), 0.25, dtype=torch.float32, device="cuda")
    solver.force(p, m, out=base, accumulate=True)
    assert np.abs(base.double().cpu().numpy() - 0.25 - acc).max() <= 1e-5 * max(np.abs(acc).max(), 1.0)
    solver.close()


def test_clustered_2M_full_size():
    box = inputs.config_box(2)
    n_mesh, rc = 128, box.r_cut
    assert abs(rc - 3.0 / n_mesh) < 1e-15
    ref = opm.pm_forces(box.pos, box.mass, n_mesh, rc, box.G)
    solver = PMSolver(n_mesh, rc, box.G)
    acc = solver.force(torch.tensor(box.pos, device="cuda"), torch.tensor(box.mass, device="cuda"))
    rms, mx = rel_err(acc.double().cpu().numpy(), ref)
    assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
    solver.close()


def test_treepm_total_through_the_library_matches_ewald():
    rng = np.random.default_rng(1)
    n, n_mesh, G = 64, 32, 1.0
    pos = rng.random((n, 3))
    mass = np.full(n, 1.0 / n)
    rc = 3.0 / n_mesh
    p, m = torch.tensor(pos, device="cuda"), torch.tensor(mass, device="cuda")
    tree = ShortRangeTree(p, m, Params(G, 0.0, rc, 0.0, 8, 8, "fp32"))
    acc = tree.force()
    PMSolver(n_mesh, rc, G).force(p, m, out=acc, accumulate=True)
    ref = ewald(pos, mass, G)
    e = np.linalg.norm(acc.double().cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.sqrt(np.mean(e ** 2)) <= 3e-2 and e.max() <= 0.1
    total_oracle = oracle.brute_force(pos, mass, G, 0.0, rc) + opm.pm_forces(pos, mass, n_mesh, rc, G)
    rms, _ = rel_err(acc.double().cpu().numpy(), total_oracle)
    assert rms <= 1e-5, rms
    tree.close()


def test_pm_errors_and_empty():
    with pytest.raises(TreeSRError):
        PMSolver(15, 0.2)                      # odd mesh
    with pytest.raises(TreeSRError):
        PMSolver(16, 0.5)                      # r_cut must be < 1/2
    s = PMSolver(16, 3 / 16)
    empty = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert s.force(empty).shape == (0, 3)
    s.close()


@pytest.mark.parametrize("name,pos,mass,n_mesh,G", cases()[::2], ids=[c[0] for c in cases()[::2]])
def test_pm_vjp_matches_oracle(name, pos, mass, n_mesh, G):
    """The PM adjoint against the oracle's (itself pinned by central
    differences): per coordinate within 1e-4 of max(|ref|, rms(ref)), the
    bound of the short-range adjoint; the one-pass call equals the two."""
    rc = 3.0 / n_mesh
    n = pos.shape[0]
    m_ref = np.full(n, 1.0 / n) if mass is None else mass
    w = inputs.cotangent(n, 99)
    ref = opm.pm_vjp(pos, m_ref, n_mesh, rc, G, w.astype(np.float64))
    solver = PMSolver(n_mesh, rc, G)
    p = torch.tensor(pos, device="cuda")
    m = None if mass is None else torch.tensor(mass, device="cuda")
    cot = torch.tensor(w, device="cuda")
    g = solver.vjp(p, m, cot).cpu().numpy()
    scale = np.sqrt(np.mean(ref ** 2))
    bad = np.abs(g - ref) > 1e-4 * np.maximum(np.abs(ref), scale)
    assert not bad.any(), (int(bad.sum()), float(np.abs(g - ref).max() / scale))
    acc1, g1 = solver.force_vjp(p, m, cot)
    # the same kernels, but the FP32 atomic adds into the mass and cotangent
    # meshes land in another order, which the potential solve carries to the
    # gradient at a few 1e-6 of its scale
    assert np.abs(g1.cpu().numpy() - g).max() <= 3e-5 * scale
    assert torch.allclose(acc1, solver.force(p, m), rtol=0, atol=1e-6 * float(acc1.abs().max()))
    base = torch.full((n, 3), 2.0, dtype=torch.float64, device="cuda")
    solver.vjp(p, m, cot, out=base, accumulate=True)
    assert np.abs(base.cpu().numpy() - 2.0 - g).max() <= 3e-5 * scale
    solver.close()


def test_captured_treepm_step_equals_direct_calls():
    """The whole TreePM step (rebuild, short-range forces and adjoint, PM
    forces and adjoint added) replayed from one CUDA graph equals the direct
    calls (up to the order of atomic adds)."""
    from paper_1211_4406_gb300.api import CapturedStep
    box = inputs.config_box(2, n_override=2 ** 15)
    n_mesh = 32
    rc = 3.0 / n_mesh
    p = torch.tensor(box.pos, device="cuda")
    m = torch.tensor(box.mass, device="cuda")
    cot = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device="cuda")
    tree = ShortRangeTree(p, m, Params(box.G, box.eps, rc, box.theta, 64, 8, "fp32"))
    pm = PMSolver(n_mesh, rc, box.G)
    a_ref, g_ref = tree.force_vjp(cot)
    pm.force_vjp(p, m, cot, acc=a_ref, grad=g_ref, accumulate=True)
    a_ref, g_ref = a_ref.clone(), g_ref.clone()
    acc = torch.empty_like(a_ref)
    grad = torch.empty_like(g_ref)
    step = CapturedStep(tree, p, m, cot, acc, grad, pm=pm)
    acc.zero_()
    grad.zero_()
    step.replay()
    torch.cuda.synchronize()
    assert tree.status() == 0
    sa = float(a_ref.abs().max())
    assert float((acc - a_ref).abs().max()) <= 1e-5 * sa
    sg = float(g_ref.pow(2).mean().sqrt())
    assert float((grad - g_ref).abs().max()) <= 1e-4 * sg
    pm.close()
    tree.close()


def test_single_particle_feels_no_pm_force():
    """One particle anywhere: the TSC assignment and interpolation with the
    antisymmetric four-point difference conserve momentum, so m a = 0."""
    rng = np.random.default_rng(21)
    s = PMSolver(16, 3 / 16, 1.0)
    for _ in range(4):
        p = torch.tensor(rng.random((1, 3)), device="cuda")
        a = s.force(p, torch.ones(1, dtype=torch.float64, device="cuda")).double().cpu().numpy()
        # scale: the force of a unit mass at one mesh spacing, G m / h^2 = 256
        assert np.abs(a).max() <= 1e-5 * 256.0, a
    s.close()
