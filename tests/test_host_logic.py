"""Host-side logic around the kernels, on CPU: the per-box n_crit tuner
(every Params field but n_crit kept, one tuning per bucket, the cache reused),
the clock summary the bench attaches to its line, and the bench's refusal of
a kernel variant on a workload that would ignore it."""
import sys
from types import SimpleNamespace

import numpy as np
import pytest

import bench
from paper_1211_4406_gb300 import autotune
from paper_1211_4406_gb300.api import Params


def test_tune_box_keeps_every_field_but_n_crit(monkeypatch):
    seen = []

    def fake_time_step(pos, mass, params, cot, reps=3):
        seen.append(params)
        return abs(params.n_crit - 48) + 1.0            # fastest at 48

    monkeypatch.setattr(autotune, "time_step", fake_time_step)
    base = Params(G=2.0, eps=0.01, r_cut=0.1, theta=0.3, n_crit=64, n_leaf=4, precision="fp64",
                  chunked=True, xi="softened")
    best, times = autotune.tune_box(None, None, base, None, candidates=(16, 32, 48, 64))
    assert best == 48 and sorted(times) == [16, 32, 48, 64]
    assert [p.n_crit for p in seen] == [16, 32, 48, 64]
    for p in seen:
        assert (p.G, p.eps, p.r_cut, p.theta, p.n_leaf, p.precision, p.chunked, p.xi) == \
            (2.0, 0.01, 0.1, 0.3, 4, "fp64", True, "softened")
    assert base.n_crit == 64                             # the caller's Params is not changed


def test_tune_boxes_tunes_each_bucket_once_and_reuses_the_cache(monkeypatch, tmp_path):
    calls = []

    def fake_tune_box(pos, mass, prm, cot, candidates, reps):
        calls.append((pos.shape[0], prm.xi))
        return 16 * (1 + len(calls)), {}

    monkeypatch.setattr(autotune, "gpu_key", lambda: "GPU|152")
    monkeypatch.setattr(autotune, "tune_box", fake_tune_box)

    def box(n):
        return SimpleNamespace(n=n, pos=np.zeros((n, 3)), mass=np.full(n, 1.0 / n))

    boxes = [box(4096), box(4100), box(4096), box(8192)]     # 4100 rounds to the 2^12 bucket
    kinds = ["uniform", "uniform", "clustered", "uniform"]
    plain = [Params(n_crit=64)] * 4
    cache = str(tmp_path / "tune.json")
    first = autotune.tune_boxes(boxes, kinds, plain, cache_path=cache, device="cpu")
    assert len(calls) == 3                                  # (2^12, uniform), (2^12, clustered), (2^13, uniform)
    assert first[0] == first[1] and len(set(first)) == 3
    again = autotune.tune_boxes(boxes, kinds, plain, cache_path=cache, device="cpu")
    assert again == first and len(calls) == 3               # all from the cache
    soft = [Params(n_crit=64, xi="softened")] * 4           # another kernel variant: its own buckets
    autotune.tune_boxes(boxes[:1], kinds[:1], soft[:1], cache_path=cache, device="cpu")
    assert len(calls) == 4 and calls[-1] == (4096, "softened")
    keys = set(autotune.load_cache(cache))
    assert "GPU|152|n2^12|uniform" in keys and "GPU|152|n2^12|uniform|xi-softened" in keys


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_summary_uses_the_timed_region_only():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = ["0, 1200, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active"]   # before the region
    s.mark()
    s.lines += ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage",
                "0, 2055, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    clk = s.stop()
    assert clk["sm_mhz"] == 2055.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"] and clk["samples"] == 3


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler(0)
    s.first = 0
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("workload", ["batched-64", "uniform-32k", "treepm-2M"])
def test_bench_refuses_a_variant_the_workload_would_ignore(monkeypatch, workload):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload, "--xi", "softened"])
    with pytest.raises(SystemExit) as e:
        bench.main()
    assert e.value.code == 2
