"""TP_FLAG_RSQRT_REFINED, the paper's inverse square root (Sec. II-A: an
estimate refined by one third-order step) in the FP32 pair kernels, against
the oracle's version of the same variant on identical lists: forces (rms
<= 1e-6, max <= 1e-4), the adjoint (1e-4 per coordinate) and the one-pass
call, with the plain and the softened cutoff argument; the flag is refused
for FP64 trees and for batches that disagree on it.  A mistake in the
refinement (a missing third-order step leaves 1.8e-3, a wrong coefficient
~1e-5) would fail the force bounds."""
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


@pytest.mark.parametrize("xi", ["plain", "softened"])
def test_refined_root_forces_and_adjoint_match_the_oracle_variant(xi):
    box = inputs.config_box(4, n_override=32768)
    w = inputs.cotangent(box.n, box.seed + 7)
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32", xi=xi, rsqrt="refined")
    soft = xi == "softened"
    ot = oracle.OracleTree(box.pos, box.mass, box.n_leaf, box.n_crit)
    ot.lists(box.r_cut, box.theta)
    ref = ot.list_forces(box.G, box.eps, box.r_cut, xi_softened=soft, rsqrt_refined=True)
    gref = ot.list_vjp(box.G, box.eps, box.r_cut, w.astype(np.float64), xi_softened=soft, rsqrt_refined=True)
    scale = np.sqrt(np.mean(gref ** 2))
    for tile in ((2, 4), (1, 2), (4, 4)):
        t = ShortRangeTree(pos, mass, prm)
        t.set_tile(*tile)
        a = t.force().double().cpu().numpy()
        g = t.vjp(torch.tensor(w, device="cuda")).cpu().numpy()
        a2, g2 = t.force_vjp(torch.tensor(w, device="cuda"))
        t.close()
        for acc in (a, a2.double().cpu().numpy()):
            rms, mx = rel_err(acc, ref)
            assert rms <= 1e-6 and mx <= 1e-4, (tile, rms, mx)
        for grad in (g, g2.cpu().numpy()):
            bad = np.abs(grad - gref) > 1e-4 * np.maximum(np.abs(gref), scale)
            assert not bad.any(), (tile, int(bad.sum()))


def test_refined_root_refused_where_it_does_not_apply():
    pos = torch.rand((1000, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(TreeSRError):
        ShortRangeTree(pos, None, Params(r_cut=0.1, precision="fp64", rsqrt="refined"))
    with pytest.raises(TreeSRError):
        ShortRangeTree(pos, None, [Params(r_cut=0.1, rsqrt="refined"), Params(r_cut=0.1)], box_offsets=[0, 500, 1000])
