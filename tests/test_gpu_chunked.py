"""Chunked mode (bounded list memory): the walk and the pair kernels run over
windows of consecutive groups and reuse one set of list buffers.  Forced with
TP_FLAG_CHUNKED on a small box (windows of ~1/4 of the lists), it must give
the same lists statistics, bit-identical forces (each group's arithmetic does
not depend on the window it is evaluated in) and the same adjoint up to the
order of FP64 atomic additions, also after a rebuild from moved particles."""
import numpy as np
import pytest
import torch

from paper_1211_4406_gb300 import inputs
from paper_1211_4406_gb300._lib import TreeSRError
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu


def trees(box, precision):
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    p = dict(G=box.G, eps=box.eps, r_cut=box.r_cut, theta=box.theta, n_crit=64, n_leaf=8,
             precision=precision)
    return pos, mass, ShortRangeTree(pos, mass, Params(**p)), ShortRangeTree(pos, mass, Params(**p, chunked=True))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_chunked_equals_whole_lists(precision):
    box = inputs.config_box(4, n_override=2 ** 15)
    pos, mass, whole, chunk = trees(box, precision)
    sw, sc = whole.stats(), chunk.stats()
    assert sw["n_windows"] == 1 and sc["n_windows"] >= 3
    for k in ("n_nodes", "n_groups", "n_entries", "n_interactions", "max_nj"):
        assert sw[k] == sc[k], k
    assert torch.equal(whole.force(), chunk.force())
    cot = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device="cuda")
    gw, gc = whole.vjp(cot).cpu().numpy(), chunk.vjp(cot).cpu().numpy()
    scale = np.sqrt(np.mean(gw ** 2))
    assert np.abs(gw - gc).max() <= 1e-12 * scale
    # new positions: rebuild (the windows are re-planned by the next call)
    pos2 = pos + 3e-4 * torch.randn(pos.shape, dtype=pos.dtype, device="cuda",
                                     generator=torch.Generator(device="cuda").manual_seed(5))
    whole.rebuild(pos2, mass)
    chunk.rebuild(pos2, mass)
    assert torch.equal(whole.force(), chunk.force())
    assert whole.status() == 0 and chunk.status() == 0
    assert chunk.stats()["n_interactions"] == whole.stats()["n_interactions"]
    with pytest.raises(TreeSRError):
        chunk.export_lists()
    whole.close()
    chunk.close()


def test_chunked_batched_boxes():
    boxes = inputs.batched_boxes(6, scale=0.25)
    pos = torch.tensor(np.concatenate([b.pos for b in boxes]), device="cuda")
    mass = torch.tensor(np.concatenate([b.mass for b in boxes]), device="cuda")
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).tolist()
    prm = [Params(b.G, b.eps, b.r_cut, b.theta, 32, 8, "fp32") for b in boxes]
    whole = ShortRangeTree(pos, mass, prm, box_offsets=offs)
    prm[2] = Params(boxes[2].G, boxes[2].eps, boxes[2].r_cut, boxes[2].theta, 32, 8, "fp32", chunked=True)
    chunk = ShortRangeTree(pos, mass, prm, box_offsets=offs)
    assert chunk.stats()["n_windows"] > 1
    assert torch.equal(whole.force(), chunk.force())
    whole.close()
    chunk.close()


@pytest.mark.parametrize("precision,eps0", [("fp64", False), ("fp32", True)])
def test_chunked_general_kernels(precision, eps0):
    """Tiny boxes (groups spanning half the box: the integer-offset general
    kernels) and eps = 0 (the scalar FP32 kernel) through the chunked path."""
    boxes = [inputs.config_box(1, n_override=n) for n in (512, 729, 1000, 4096)]
    pos = torch.tensor(np.concatenate([b.pos for b in boxes]), device="cuda")
    mass = torch.tensor(np.concatenate([b.mass for b in boxes]), device="cuda")
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).tolist()

    def prm(chunked):
        return [Params(b.G, 0.0 if eps0 else b.eps, b.r_cut, b.theta, 32, 8, precision, chunked=chunked)
                for b in boxes]
    whole = ShortRangeTree(pos, mass, prm(False), box_offsets=offs)
    chunk = ShortRangeTree(pos, mass, prm(True), box_offsets=offs)
    assert chunk.stats()["n_windows"] > 1
    assert torch.equal(whole.force(), chunk.force())
    cot = torch.tensor(np.concatenate([inputs.cotangent(b.n, b.seed + 7) for b in boxes]), device="cuda")
    gw, gc = whole.vjp(cot).cpu().numpy(), chunk.vjp(cot).cpu().numpy()
    assert np.abs(gw - gc).max() <= 1e-12 * np.sqrt(np.mean(gw ** 2))
    whole.close()
    chunk.close()
