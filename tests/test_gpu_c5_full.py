"""Full-size validation of the throughput box, in the launch configuration
the benchmark times: N = 512^3 clustered particles (10^5 halos), r_cut =
3/512, eps = 1/25600, lists in chunked mode, forces and adjoint in one pass
(tp_short_range_force_vjp).  Sampled outputs against the oracle's O(N)
direct sums (Eq. 2 and its gradient over every particle):

- theta = 0 (every neighbour within r_cut is a particle entry): FP32 forces
  rms <= 1e-6 and max <= 1e-4, the FP32 bounds; the adjoint within 1e-4 of
  max(|ref|, rms(ref)) per coordinate;
- theta = 0.5 (the benchmark's lists): forces rms <= 5e-3 against the
  direct sum, the tree's bound.

Generating the box takes about two minutes of one CPU core, so this runs
only with TP_ONEOFF=1.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = [pytest.mark.gpu, pytest.mark.oneoff]


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def test_throughput_box_full_size_sampled():
    box = inputs.config_box(5)
    assert box.n == 512 ** 3
    w = inputs.cotangent(box.n, box.seed + 7)
    dev = torch.device("cuda")
    pos = torch.from_numpy(box.pos).to(dev)
    mass = torch.from_numpy(box.mass).to(dev)
    cot = torch.from_numpy(w).to(dev)
    idx = np.sort(np.random.default_rng(5).choice(box.n, 128, replace=False))
    ref = oracle.brute_force_sample(box.pos, box.mass, box.G, box.eps, box.r_cut, idx)
    gref = oracle.brute_vjp_sample(box.pos, box.mass, box.G, box.eps, box.r_cut, w.astype(np.float64), idx)
    report = {}
    for theta in (0.0, box.theta):
        t = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, theta, box.n_crit, box.n_leaf, "fp32"))
        acc, grad = t.force_vjp(cot)
        st = t.stats()
        assert t.status() == 0 and st["n_windows"] > 1
        rms, mx = rel_err(acc[torch.from_numpy(idx).to(dev)].double().cpu().numpy(), ref)
        report[theta] = (rms, mx, st["n_windows"], st["n_entries"])
        if theta == 0.0:
            assert rms <= 1e-6 and mx <= 1e-4, (rms, mx)
            g = grad[torch.from_numpy(idx).to(dev)].cpu().numpy()
            scale = np.sqrt(np.mean(gref ** 2))
            bad = np.abs(g - gref) > 1e-4 * np.maximum(np.abs(gref), scale)
            assert not bad.any(), (int(bad.sum()), float(np.abs(g - gref).max() / scale))
        else:
            assert rms <= 5e-3, (rms, mx)
        del acc, grad
        t.close()
        torch.cuda.empty_cache()
    print("throughput box, sampled vs direct sum:", report)
