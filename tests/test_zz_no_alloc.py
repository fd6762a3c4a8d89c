"""tp_short_range_force_noalloc, the entry point for callers that must not let
the library allocate device memory (their device memory comes from their own
pool, or an allocation's implicit synchronisation is too costly for them).

Its result is checked through the C-ABI on two calls in a row that reuse the
one static scratch array, with the FP32 tolerance of the other parity tests,
against the tree entry point (tp_build_tree + tp_short_range_force at
theta = 0, the same exact cutoff sum) and against the oracle's FP64 direct
sum; the default-mass path (mass = NULL, every mass 1/n) against the tree
entry point with mass = None; and its refusals: sizes beyond its array,
parameters it does not take, and non-finite positions.  Collected last on
purpose, so that a run stopping at the first failure has run everything else
first."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_1211_4406_gb300 import _lib, inputs
from paper_1211_4406_gb300.api import Params, ShortRangeTree

pytestmark = pytest.mark.gpu

FP32_RMS, FP32_MAX = 1e-6, 1e-4
TP_ERR_INVALID_ARG, TP_ERR_NONFINITE = -1, -6


def rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def call_noalloc(pos, mass, prm, acc, flags=0):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = prm.c()
    p.flags = flags
    return _lib.load().tp_short_range_force_noalloc(
        C.c_void_p(pos.data_ptr()), C.c_void_p(mass.data_ptr()) if mass is not None else None,
        pos.shape[0], C.byref(p), C.c_void_p(acc.data_ptr()), stream)


def test_noalloc_matches_tree_entry_point_and_direct_sum_twice():
    boxes = [inputs.config_box(4, n_override=6000),                       # clustered
             inputs.Box("uniform", *inputs.uniform_box(20000, 99), 1.3, 1e-3, 0.11, 0.0)]
    for box in boxes:                                                    # two calls in a row
        pos = torch.tensor(box.pos, device="cuda")
        mass = torch.tensor(box.mass, device="cuda")
        prm = Params(box.G, box.eps, box.r_cut, 0.0, 64, 8, "fp32")
        acc = torch.full((box.n, 3), float("nan"), dtype=torch.float32, device="cuda")
        assert call_noalloc(pos, mass, prm, acc) == 0
        torch.cuda.synchronize()
        got = acc.double().cpu().numpy()
        tree = ShortRangeTree(pos, mass, prm)
        ref_tree = tree.force().double().cpu().numpy()
        tree.close()
        rms, mx = rel_err(got, ref_tree)
        assert rms <= FP32_RMS and mx <= FP32_MAX, (box.name, "vs tree", rms, mx)
        ref = oracle.brute_force(box.pos, box.mass, box.G, box.eps, box.r_cut)
        rms, mx = rel_err(got, ref)
        assert rms <= FP32_RMS and mx <= FP32_MAX, (box.name, "vs direct sum", rms, mx)


def test_noalloc_default_masses():
    pos_h, _ = inputs.uniform_box(5000, 7)
    pos = torch.tensor(pos_h, device="cuda")
    prm = Params(1.0, 1e-3, 0.12, 0.0, 64, 8, "fp32")
    acc = torch.full((pos.shape[0], 3), float("nan"), dtype=torch.float32, device="cuda")
    assert call_noalloc(pos, None, prm, acc) == 0
    torch.cuda.synchronize()
    tree = ShortRangeTree(pos, None, prm)
    ref = tree.force().double().cpu().numpy()
    tree.close()
    rms, mx = rel_err(acc.double().cpu().numpy(), ref)
    assert rms <= FP32_RMS and mx <= FP32_MAX, (rms, mx)


def test_noalloc_refusals():
    _lib.load()
    big = 65536 + 1
    pos = torch.rand((big, 3), dtype=torch.float64, device="cuda")
    acc = torch.empty((big, 3), dtype=torch.float32, device="cuda")
    assert call_noalloc(pos, None, Params(r_cut=0.05), acc) == TP_ERR_INVALID_ARG
    assert call_noalloc(pos[:0], None, Params(r_cut=0.05), acc[:0]) == 0
    small, out = pos[:100], acc[:100]
    assert call_noalloc(small, None, Params(r_cut=0.05), out, flags=2) == TP_ERR_INVALID_ARG
    assert call_noalloc(small, None, Params(r_cut=0.05, precision="fp64"), out) == TP_ERR_INVALID_ARG
    assert call_noalloc(small, None, Params(r_cut=0.5), out) == TP_ERR_INVALID_ARG
    assert call_noalloc(small, None, Params(r_cut=0.05, eps=-1.0), out) == TP_ERR_INVALID_ARG
    host = torch.rand((100, 3), dtype=torch.float64)
    assert call_noalloc(host, None, Params(r_cut=0.05), out) == TP_ERR_INVALID_ARG
    # a non-finite position is refused and the output is left alone; the
    # next call on good positions runs normally
    bad = small.clone()
    bad[17, 1] = float("nan")
    out.fill_(3.0)
    assert call_noalloc(bad, None, Params(r_cut=0.05), out) == TP_ERR_NONFINITE
    torch.cuda.synchronize()
    assert bool((out == 3.0).all())
    bad[17, 1] = float("inf")
    assert call_noalloc(bad, None, Params(r_cut=0.05), out) == TP_ERR_NONFINITE
    assert call_noalloc(small, None, Params(r_cut=0.05), out) == 0
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
