"""Group-size autotuner for the batched persistent launch.

For every box the group size n_crit (Barnes' <N_i>, Sec. II) is chosen among
candidates by timing the whole step (rebuild, force, adjoint) on the GPU; the
choice is cached in JSON keyed by GPU name, SM count, particle-count bucket
(log2) and the box kind, so boxes of the same shape reuse it.
"""
from __future__ import annotations

import json
import math
import os

import torch

from .api import Params, ShortRangeTree

CANDIDATES = (16, 24, 32, 48, 64, 96, 128, 192, 256)


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "treepm_sr", "autotune.json")


def gpu_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def bucket_key(n: int, kind: str) -> str:
    return f"{gpu_key()}|n2^{int(round(math.log2(max(n, 1))))}|{kind}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_step(pos, mass, params: Params, cot, reps: int = 3) -> float:
    """Median milliseconds of rebuild + force + adjoint for one box."""
    t = ShortRangeTree(pos, mass, params)
    acc = torch.empty((t.n, 3), dtype=t.acc_dtype, device=pos.device)
    grad = torch.empty((t.n, 3), dtype=torch.float64, device=pos.device)
    ts = []
    for r in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        t.rebuild(pos, mass)
        t.force(acc)
        t.vjp(cot, grad)
        b.record()
        b.synchronize()
        if r:
            ts.append(a.elapsed_time(b))
    t.close()
    ts.sort()
    return ts[len(ts) // 2]


def tune_box(pos, mass, base: Params, cot, candidates=CANDIDATES, reps: int = 3) -> tuple[int, dict]:
    times = {}
    for c in candidates:
        p = Params(base.G, base.eps, base.r_cut, base.theta, c, base.n_leaf, base.precision)
        times[c] = time_step(pos, mass, p, cot, reps)
    best = min(times, key=times.get)
    return best, times


def tune_boxes(boxes, kinds, base_params, cache_path: str | None = None, candidates=CANDIDATES,
               reps: int = 3, device="cuda") -> list[int]:
    """n_crit per box (list), tuning each (size bucket, kind) once."""
    cache_path = cache_path or default_cache_path()
    cache = load_cache(cache_path)
    out = []
    for box, kind, prm in zip(boxes, kinds, base_params):
        key = bucket_key(box.n, kind)
        if key not in cache:
            pos = torch.tensor(box.pos, device=device)
            mass = torch.tensor(box.mass, device=device)
            cot = torch.randn((box.n, 3), dtype=torch.float32, device=device,
                              generator=torch.Generator(device=device).manual_seed(box.n))
            best, times = tune_box(pos, mass, prm, cot, candidates, reps)
            cache[key] = {"n_crit": best, "ms": {str(k): v for k, v in times.items()}}
        out.append(int(cache[key]["n_crit"]))
    save_cache(cache_path, cache)
    return out
