"""Run the hot path once or a few times on a synthetic clustered box, for
profilers (ncu launch lists and single-kernel captures).

  python -m paper_1211_4406_gb300.profile_step [--n N] [--steps K] [--what step|force|vjp]

--n 2097152 is the benchmark workload (128^3 particles, 2000 NFW halos,
r_cut = 3/128); smaller n keeps the recipe (halo count, r_cut and eps scale
with n).  The allocating build runs first; each step is rebuild + force +
adjoint (or only the force / only the adjoint).
"""
from __future__ import annotations

import argparse

import torch

from . import build as _build
from . import inputs
from .api import Params, ShortRangeTree


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128 ** 3)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--what", default="step", choices=["step", "force", "vjp"])
    args = ap.parse_args()
    _build.build()
    box = inputs.config_box(2, n_override=args.n)
    pos = torch.tensor(box.pos, device="cuda")
    mass = torch.tensor(box.mass, device="cuda")
    cot = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device="cuda")
    t = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit,
                                         box.n_leaf, "fp32"))
    acc = torch.empty((box.n, 3), dtype=torch.float32, device="cuda")
    grad = torch.empty((box.n, 3), dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        if args.what == "step":
            t.rebuild(pos, mass)
        if args.what in ("step", "force"):
            t.force(acc)
        if args.what in ("step", "vjp"):
            t.vjp(cot, grad)
    torch.cuda.synchronize()
    st = t.stats()
    print(f"status={t.status()} n={st['n']} groups={st['n_groups']} entries={st['n_entries']} "
          f"interactions={st['n_interactions']}")
    t.close()


if __name__ == "__main__":
    main()
