"""The Python binding refuses buffers that the library would read or write
past their end (wrong length, shape or dtype) before the call reaches the
library, and the tree stays usable afterwards."""
import pytest
import torch

from paper_1211_4406_gb300.api import Params, PMSolver, ShortRangeTree, axpy, scale

pytestmark = pytest.mark.gpu


def test_wrong_sizes_and_dtypes_are_refused_before_the_library():
    torch.manual_seed(3)
    n = 256
    dev = torch.device("cuda")
    pos = torch.rand((n, 3), dtype=torch.float64, device=dev)
    mass = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    cot = torch.randn((n, 3), dtype=torch.float32, device=dev)
    prm = Params(G=1.0, eps=1e-3, r_cut=0.2, theta=0.5, n_crit=16)

    with pytest.raises(ValueError):
        ShortRangeTree(pos, mass[:-1], prm)                    # too few masses
    with pytest.raises(TypeError):
        ShortRangeTree(pos, mass.float(), prm)                 # float32 masses
    t = ShortRangeTree(pos, mass, prm)
    with pytest.raises(ValueError):
        t.rebuild(pos, mass[:-1])
    with pytest.raises(ValueError):
        t.refit(pos, mass.view(n, 1))
    with pytest.raises(ValueError):
        t.force(out=torch.empty((n - 1, 3), dtype=torch.float32, device=dev))
    with pytest.raises(ValueError):
        t.vjp(cot[:-1])
    with pytest.raises(ValueError):
        t.vjp(cot, out=torch.empty((n, 3), dtype=torch.float32, device=dev))
    with pytest.raises(ValueError):
        t.force_vjp(cot[:, :2])
    with pytest.raises(ValueError):
        t.force_vjp(cot, grad=torch.empty((n, 3), dtype=torch.float32, device=dev))
    a, g = t.force_vjp(cot.double())                           # any float cotangent is converted
    a2 = t.force()
    torch.cuda.synchronize()
    assert t.status() == 0 and bool(torch.isfinite(g).all())
    # the one-pass and the separate forward sum the FP32 tiles in another order
    assert float((a - a2).abs().max()) <= 1e-4 * float(a2.abs().max())
    t.close()

    pm = PMSolver(16, 3 / 16)
    with pytest.raises(ValueError):
        pm.force(pos, mass[:-1])
    with pytest.raises(ValueError):
        pm.vjp(pos, mass, cot[:-1])
    with pytest.raises(ValueError):
        pm.force_vjp(pos, mass, cot, acc=torch.empty((n, 2), dtype=torch.float32, device=dev))
    assert pm.force(pos, mass).shape == (n, 3)
    pm.close()

    y = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        axpy(y, cot[:-1], 1.0)
    with pytest.raises(TypeError):
        axpy(y, cot.cpu(), 1.0)
    with pytest.raises(TypeError):
        scale(y, cot, 1.0)                                     # x must be float64
    with pytest.raises(ValueError):
        scale(y[:-1], y, 1.0)
    axpy(y, cot, 2.0)
    torch.cuda.synchronize()
    assert torch.equal(y, 2.0 * cot.double())


def test_calls_on_a_side_stream_match_the_current_stream():
    """A call given another stream waits for the binding's conversions on the
    current stream and keeps their memory alive: forces and the adjoint of a
    float64 cotangent (converted by the binding) on a side stream equal those
    on the current stream (the forces bit for bit), and so does the PM force
    up to the order of its FP32 mass-assignment atomics."""
    torch.manual_seed(5)
    n = 4096
    dev = torch.device("cuda")
    pos = torch.rand((n, 3), dtype=torch.float64, device=dev)
    mass = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    cot = torch.randn((n, 3), dtype=torch.float64, device=dev)
    prm = Params(G=1.0, eps=1e-3, r_cut=0.1, theta=0.5, n_crit=32)
    t = ShortRangeTree(pos, mass, prm)
    a0, g0 = t.force(), t.vjp(cot)
    pm = PMSolver(32, 0.1, 1.0)
    p0 = pm.force(pos, mass)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for _ in range(3):
        t.rebuild(pos.clone(), mass.clone(), stream=side)   # temporaries freed at once on this side
        a1 = t.force(stream=side)
        g1 = t.vjp(cot * 1.0, stream=side)
        p1 = pm.force(pos.clone(), mass, stream=side)
        side.synchronize()
        assert torch.equal(a0, a1)
        assert float((p0 - p1).abs().max()) <= 1e-5 * float(p0.abs().max())
        assert float((g0 - g1).abs().max()) <= 1e-12 * float(g0.abs().max())
    t.close()
    pm.close()
