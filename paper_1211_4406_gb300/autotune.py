"""Autotuner for the group size and the tile shape of the pair kernels.

For every box the group size n_crit (Barnes' <N_i>, Sec. II) is chosen among
candidates by timing the whole step (rebuild, force, adjoint) on the GPU; the
choice is cached in JSON keyed by GPU name, SM count, particle-count bucket
(log2) and the box kind, so boxes of the same shape reuse it.  For a built
tree (one box or a whole batch) the tile shape -- group particles per thread
of the forward kernel, list entries per thread of the adjoint kernel -- is
chosen the same way on the tree itself -- the forward shape by timing the
force call, the adjoint shape by timing the one-pass forces and adjoint --
and cached under a caller-given key.
"""
from __future__ import annotations

import dataclasses
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


def bucket_key(n: int, kind: str, params: Params | None = None) -> str:
    """Tuning bucket of a box: GPU, size to the nearest power of two, kind,
    and the kernel variant where it is not the default (FP32, plain xi)."""
    key = f"{gpu_key()}|n2^{int(round(math.log2(max(n, 1))))}|{kind}"
    if params is not None and params.precision != "fp32":
        key += f"|{params.precision}"
    if params is not None and params.xi != "plain":
        key += f"|xi-{params.xi}"
    return key


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
        p = dataclasses.replace(base, n_crit=c)     # every other field (precision, xi, chunked) kept
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
        key = bucket_key(box.n, kind, prm)
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


def tune_tile(tree: ShortRangeTree, pos, mass, cot, key: str | None = None, cache_path: str | None = None,
              fwd_choices=(2, 1, 4), adj_choices=(4, 2, 8), reps: int = 5) -> tuple[int, int]:
    """Tile shape of `tree` (set on it and returned): group particles per
    thread of the forward kernel, timed on the force call, and list entries
    per thread of the adjoint kernel, timed on the one-pass forces + adjoint
    call; each the choice with the shortest median.  With a key the choice is
    cached and reused for trees of the same workload."""
    cache_path = cache_path or default_cache_path()
    cache = load_cache(cache_path)
    ck = f"{gpu_key()}|tile|{key}" if key else None
    if ck and ck in cache:
        best = tuple(cache[ck]["tile"])
        tree.set_tile(*best)
        return best
    acc = torch.empty((tree.n, 3), dtype=tree.acc_dtype, device=pos.device)
    grad = torch.empty((tree.n, 3), dtype=torch.float64, device=pos.device)
    tree.rebuild(pos, mass)

    def medians_ms(choices, set_choice, fn):
        """Median event time of fn for every choice, the choices interleaved
        round by round (one untimed round first), so that a drift of the
        clocks or of the caches over the tuning does not favour one."""
        ts = {c: [] for c in choices}
        for r in range(reps + 1):
            for c in choices:
                set_choice(c)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                b.synchronize()
                if r:
                    ts[c].append(a.elapsed_time(b))
        return {c: sorted(v)[len(v) // 2] for c, v in ts.items()}

    fwd_ms = medians_ms(fwd_choices, lambda f: tree.set_tile(f, adj_choices[0]), lambda: tree.force(acc))
    best_f = min(fwd_ms, key=fwd_ms.get)
    adj_ms = medians_ms(adj_choices, lambda e: tree.set_tile(best_f, e), lambda: tree.force_vjp(cot, acc, grad))
    best = (best_f, min(adj_ms, key=adj_ms.get))
    tree.set_tile(*best)
    if ck:
        cache[ck] = {"tile": list(best), "forward_ms": {str(k): v for k, v in fwd_ms.items()},
                     "one_pass_ms": {str(k): v for k, v in adj_ms.items()}}
        save_cache(cache_path, cache)
    return best
