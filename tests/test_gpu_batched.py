"""The batched persistent launch: 64 independent boxes in one tree, the whole
step captured in one CUDA graph, group sizes from the autotuner; every box
checked against its own oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import autotune, inputs
from paper_1211_4406_gb300.api import CapturedStep, Params, ShortRangeTree

pytestmark = pytest.mark.gpu


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def test_graph_captured_batched_step(tmp_path):
    boxes = inputs.batched_boxes(64, scale=0.1)
    kinds = ["uniform" if b % 2 == 0 else "clustered" for b in range(64)]
    base = [Params(b.G, b.eps, b.r_cut, b.theta, 64, 8, "fp32") for b in boxes]
    ncrit = autotune.tune_boxes(boxes, kinds, base, cache_path=str(tmp_path / "tune.json"),
                                candidates=(32, 64, 128), reps=1)
    assert all(c in (32, 64, 128) for c in ncrit)
    assert autotune.load_cache(str(tmp_path / "tune.json"))
    prm = [Params(b.G, b.eps, b.r_cut, b.theta, c, 8, "fp32") for b, c in zip(boxes, ncrit)]
    pos = torch.tensor(np.concatenate([b.pos for b in boxes]), device="cuda")
    mass = torch.tensor(np.concatenate([b.mass for b in boxes]), device="cuda")
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    cot = torch.tensor(np.concatenate([inputs.cotangent(b.n, b.seed + 7) for b in boxes]), device="cuda")
    tree = ShortRangeTree(pos, mass, prm, box_offsets=offs.tolist())
    acc = torch.empty((tree.n, 3), dtype=torch.float32, device="cuda")
    grad = torch.empty((tree.n, 3), dtype=torch.float64, device="cuda")
    step = CapturedStep(tree, pos, mass, cot, acc, grad)
    acc.zero_()
    step.replay()
    torch.cuda.synchronize()
    assert tree.status() == 0
    a = acc.double().cpu().numpy()
    g = grad.cpu().numpy()
    for k, (b, c) in enumerate(zip(boxes, ncrit)):
        sl = slice(offs[k], offs[k + 1])
        ot = oracle.OracleTree(b.pos, b.mass, 8, c)
        ot.lists(b.r_cut, b.theta)
        rms, mx = rel_err(a[sl], ot.list_forces(b.G, b.eps, b.r_cut))
        assert rms <= 1e-6 and mx <= 1e-4, (k, rms, mx)
        if k % 8 == 1:
            gref = ot.list_vjp(b.G, b.eps, b.r_cut, inputs.cotangent(b.n, b.seed + 7).astype(np.float64))
            sc = np.sqrt(np.mean(gref ** 2))
            assert np.all(np.abs(g[sl] - gref) <= 1e-4 * np.maximum(np.abs(gref), sc)), k
    # moving the particles a little and replaying re-walks the same graph
    pos += 1e-5
    step.replay()
    torch.cuda.synchronize()
    assert tree.status() == 0
    b = boxes[3]
    ot = oracle.OracleTree(b.pos + 1e-5, b.mass, 8, ncrit[3])
    ot.lists(b.r_cut, b.theta)
    rms, mx = rel_err(acc.double().cpu().numpy()[offs[3]:offs[4]], ot.list_forces(b.G, b.eps, b.r_cut))
    assert rms <= 1e-6 and mx <= 1e-4
    tree.close()
