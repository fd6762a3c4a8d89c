"""tp_short_range_force_noalloc, the entry point for callers that must not let
the library allocate device memory (their device memory comes from their own
pool, or an allocation's implicit synchronisation is too costly for them).
Its result is checked through the C-ABI against the tree entry point
(tp_build_tree + tp_short_range_force with theta = 0, which is the same exact
cutoff sum) on two calls in a row that reuse the one static scratch array,
with the FP32 tolerance of the other parity tests.  Collected last on purpose,
so that a run stopping at the first failure has run everything else first."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1211_4406_gb300 import _lib, inputs
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu

FP32_RMS, FP32_MAX = 1e-6, 1e-4


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def call_noalloc(pos, mass, prm, acc):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = prm.c()
    return _lib.load().tp_short_range_force_noalloc(
        C.c_void_p(pos.data_ptr()), C.c_void_p(mass.data_ptr()) if mass is not None else None,
        pos.shape[0], C.byref(p), C.c_void_p(acc.data_ptr()), stream)


def test_noalloc_matches_tree_entry_point_twice():
    boxes = [inputs.config_box(4, n_override=6000),                       # clustered
             inputs.Box("uniform", *inputs.uniform_box(20000, 99), 1.3, 1e-3, 0.11, 0.0)]
    for box in boxes:                                                    # two calls in a row
        pos = torch.tensor(box.pos, device="cuda")
        mass = torch.tensor(box.mass, device="cuda")
        prm = Params(box.G, box.eps, box.r_cut, 0.0, 64, 8, "fp32")
        acc = torch.full((box.n, 3), float("nan"), dtype=torch.float32, device="cuda")
        assert call_noalloc(pos, mass, prm, acc) == 0
        torch.cuda.synchronize()
        ref = ShortRangeTree(pos, mass, prm).force().double().cpu().numpy()
        rms, mx = rel_err(acc.double().cpu().numpy(), ref)
        assert rms <= FP32_RMS and mx <= FP32_MAX, (box.name, rms, mx)


def test_noalloc_rejects_sizes_beyond_its_array():
    _lib.load()
    big = 65536 + 1
    pos = torch.rand((big, 3), dtype=torch.float64, device="cuda")
    acc = torch.empty((big, 3), dtype=torch.float32, device="cuda")
    assert call_noalloc(pos, None, Params(r_cut=0.05), acc) == -1
    assert call_noalloc(pos[:0], None, Params(r_cut=0.05), acc[:0]) == 0
