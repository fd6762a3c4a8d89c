"""Run the hot path once or a few times on a synthetic clustered box, for
profilers (ncu launch lists and single-kernel captures).

  python -m paper_1211_4406_gb300.profile_step [--n N] [--steps K] [--what step|force|vjp|fused|all] [--tile F,A]

--n 2097152 is the benchmark workload (128^3 particles, 2000 NFW halos,
r_cut = 3/128); smaller n keeps the recipe (halo count, r_cut and eps scale
with n).  The allocating build runs first; each step is rebuild + force +
adjoint (step), only the force or only the adjoint, rebuild + the one-pass
force and adjoint (fused), or rebuild + all three (all).

  python -m paper_1211_4406_gb300.profile_step --record-traffic CSV --n N --entries E

reads an ncu CSV of dram__bytes_read.sum / dram__bytes_write.sum /
gpu__time_duration.sum for the pair kernels (taken on this command with --n N,
whose tree has E list entries) and writes the per-launch DRAM traffic, with
the digest of the device code it was measured on, to
profiles/kernel_traffic.json.  The capture is taken on a smaller box of the
clustered recipe (a few GB on the device, so that the multi-metric replay
stays short); the pair kernels stream each list entry's record once per
launch, so their traffic scales with the entry count, and traffic_for
scales the record to the tree it is asked about.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os

from . import build as _build
from . import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "kernel_traffic.json")
TRAFFIC_KERNELS = ("k_pair_packed", "k_vjp_fused", "k_vjp_epack")


def kernel_key(name: str) -> str:
    """A kernel's name with template arguments in one spelling (ncu prints
    bool arguments as 0/1)."""
    return name.replace(" ", "").replace("true", "1").replace("false", "0")


def kernel_source_digest() -> str:
    """SHA-256 of the pair kernels' device code: the shared header and the
    part of tp_pair.cu before its host launch functions."""
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    h = hashlib.sha256()
    h.update(open(os.path.join(csrc, "tp_common.cuh"), "rb").read())
    src = open(os.path.join(csrc, "tp_pair.cu"), "rb").read()
    cut = src.find(b"\nnamespace tp {")
    h.update(src if cut < 0 else src[:cut])
    return h.hexdigest()


# ncu's metric units, as multiples of a byte or a nanosecond
UNIT_SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12,
              "ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
              "s": 1e9, "second": 1e9}


def record_traffic(csv_path: str, n: int, out_path: str | None = None, entries: int | None = None) -> dict:
    """Per-launch DRAM bytes and ncu time of the pair kernels from an ncu CSV
    (one row per launch and metric), written to `out_path` (default: the
    committed traffic record), with the particle count n and the list entry
    count of the captured tree.  Values are scaled by their unit column; an
    unknown unit raises ValueError."""
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[hi]
    ki, mi, ni = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Name")
    ui = hdr.index("Metric Unit") if "Metric Unit" in hdr else None
    per = {}
    for r in rows[hi + 1:]:
        if len(r) <= mi:
            continue
        name = kernel_key(r[ki].split("(")[0].replace("<unnamed>::", "").replace("void ", ""))
        if name.split("<")[0] not in TRAFFIC_KERNELS:
            continue
        unit = r[ui] if ui is not None else ""
        if unit and unit not in UNIT_SCALE:
            raise ValueError(f"unknown ncu unit {unit!r} for {r[ni]}")
        d = per.setdefault((name, r[0]), {})
        d[r[ni]] = float(r[mi].replace(",", "")) * UNIT_SCALE.get(unit, 1.0)
    out = {}
    for (name, _), d in per.items():
        k = out.setdefault(name, {"launches": 0, "dram_bytes": 0.0, "ns": 0.0})
        k["launches"] += 1
        k["dram_bytes"] += d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
        k["ns"] += d.get("gpu__time_duration.sum", 0.0)
    rec = {"recipe": "clustered", "n": n, "entries": entries,
           "digest": kernel_source_digest(),
           "kernels": {k: {"bytes_per_launch": v["dram_bytes"] / v["launches"],
                           "ncu_ms_per_launch": v["ns"] / v["launches"] / 1e6}
                       for k, v in out.items()},
           "command": ("ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                       "--clock-control none -k regex:\"k_pair_packed|k_vjp_fused|k_vjp_epack\" -c 3 --csv --log-file "
                       f"<csv> python -m paper_1211_4406_gb300.profile_step --n {n} --steps 1 --what all --tile 2,8")}
    out_path = out_path or TRAFFIC_JSON
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def traffic_for(kernel: str, entries: int, recipe: str = "clustered", path: str | None = None):
    """DRAM bytes per launch of `kernel` (its name with template arguments, as
    ncu prints it) on a tree of the input recipe `recipe` with `entries` list
    entries: the captured bytes scaled by entries / the captured tree's
    entries.  None when no capture exists for that recipe or the device code
    has changed since it was taken."""
    try:
        rec = json.load(open(path or TRAFFIC_JSON))
    except (OSError, ValueError):
        return None
    if rec.get("recipe") != recipe or rec.get("digest") != kernel_source_digest() or not rec.get("entries"):
        return None
    k = rec.get("kernels", {}).get(kernel_key(kernel))
    if k is None:
        return None
    return k.get("bytes_per_launch") * float(entries) / float(rec["entries"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128 ** 3)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--what", default="step", choices=["step", "force", "vjp", "fused", "all", "treepm"],
                    help="treepm: rebuild + short-range force + PM force on the mesh of r_cut = 3 spacings")
    ap.add_argument("--record-traffic", metavar="CSV")
    ap.add_argument("--entries", type=int, help="list entries of the captured tree (printed by the run)")
    ap.add_argument("--tile", default="2,8", help="forward particles and adjoint entries per thread "
                    "(tp_tree_set_tile; 2,8 is the shape the autotuner picks for the clustered recipe)")
    args = ap.parse_args()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic, args.n, entries=args.entries)))
        return
    import torch

    from .api import Params, PMSolver, ShortRangeTree
    _build.build()
    box = inputs.config_box(2, n_override=args.n)
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    cot = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device="cuda")
    t = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit,
                                         box.n_leaf, "fp32"))
    t.set_tile(*(int(v) for v in args.tile.split(",")))
    acc = torch.empty((box.n, 3), dtype=torch.float32, device="cuda")
    grad = torch.empty((box.n, 3), dtype=torch.float64, device="cuda")
    pm = PMSolver(int(round(3.0 / box.r_cut)), box.r_cut, box.G) if args.what == "treepm" else None
    for _ in range(args.steps):
        if pm is not None:
            t.rebuild(pos, mass)
            t.force(acc)
            pm.force(pos, mass, out=acc, accumulate=True)
            continue
        if args.what in ("step", "fused", "all"):
            t.rebuild(pos, mass)
        if args.what in ("step", "force", "all"):
            t.force(acc)
        if args.what in ("step", "vjp", "all"):
            t.vjp(cot, grad)
        if args.what in ("fused", "all"):
            t.force_vjp(cot, acc, grad)
    torch.cuda.synchronize()
    st = t.stats()
    print(f"status={t.status()} n={st['n']} groups={st['n_groups']} entries={st['n_entries']} "
          f"interactions={st['n_interactions']}")
    t.close()


if __name__ == "__main__":
    main()
