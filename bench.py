"""Benchmark of the short-range TreePM path on GB300.

One step = the whole hot path on one synthetic box: tree build (keys, sort,
octree, monopoles, groups, interaction lists), the FP32 force (Eq. 2 on the
lists) and its adjoint (VJP with a fixed cotangent), the last two in one pass
over the lists (tp_short_range_force_vjp; the same step with separate force
and adjoint calls is timed beside it).  The workload is the FP32-precision
clustered box: N = 128^3 = 2,097,152 particles, 70 % in 2000 NFW halos,
r_cut = 3/128, eps = 1/6400, theta = 0.5, n_crit = 64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = short-range interactions per second, counting
each (i, list entry) pair of the forward pass and of the adjoint pass once
(interactions = sum over groups of n_i * n_j, the paper's count).  With N > 1
every rank runs an independent replica of the box, so scaling is weak and
value sums the ranks' interactions over the slowest rank's time; the batched
workload (--workload batched-64) shares its 64 boxes among the ranks instead,
and domain.DomainShortRange splits one box over ranks (tested on gloo ranks).
--impl reference times the CPU FP64 oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "short-range interactions/s (FP32 forward + adjoint, clustered 2M box)"
UNIT = "interactions/s"
# Algorithmic FP32 operations per interaction as evaluated (FMA = 2, rsqrt and
# sqrt = 1 each, clamps and masks not counted): the forward term of Eq. 2 with
# Eq. 3, and its vector-Jacobian product (both cutoff polynomials, phi and psi,
# d.w, the 3-vector for the list entry and the sums for the particle).
FLOPS_PER_INTERACTION = 42
VJP_FLOPS_PER_INTERACTION = 76
FUSED_FLOPS_PER_INTERACTION = 82   # the adjoint's 76 + the forward's a += alpha d (3 FMA)
PAPER_FLOPS_PER_INTERACTION = 51 # the paper's convention (Sec. II-A)
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0      # GB300's maximum SM clock; the clock sampler's reading replaces it


def fp32_peak(dev, clk=None):
    """Nominal FP32 peak of this GPU (FLOP/s) and its basis: SMs as the device
    reports them x 128 FP32 lanes x 2 (an FMA) x the maximum SM clock that
    nvidia-smi reports during the run (GB300's 2070 MHz if it reported none)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or SM_MAX_MHZ
    basis = f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz (maximum SM clock)"
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6, basis
CONFIG_K = 2


def workload_config(paper_regime: bool = False):
    if paper_regime:
        return {"workload": "paper-regime-2M", "n": 128 ** 3, "halos": 2000, "r_cut": "7.5/128",
                "eps": "1/6400", "theta": 0.5, "n_crit": 192, "n_leaf": 8, "seed": 14408,
                "l2": "flushed (256 MiB write) before every timed step",
                "why": "the paper's group size (Table I: <N_i> ~ 115) and r_cut = 7.5 mean spacings (its "
                       "4096^3 PM mesh for 10240^3 particles); its <N_j> ~ 2300 is not reached: a group box "
                       "of ~115 particles is wider than r_cut, so no monopole lies wholly inside r_cut"}
    return {"workload": "clustered-2M", "n": 128 ** 3, "halos": 2000, "r_cut": "3/128",
            "eps": "1/6400", "theta": 0.5, "n_crit": 64, "n_leaf": 8, "seed": 14408,
            "l2": "flushed (256 MiB write) before every timed step"}


def bench_box(paper_regime: bool = False):
    """The clustered 2M box; in the paper's regime with r_cut = 7.5/128 and
    n_crit = 192 (<N_i> = 109, Table I: ~115) instead of 3/128 and 64."""
    from paper_1211_4406_gb300 import inputs
    box = inputs.config_box(CONFIG_K)
    if paper_regime:
        box.r_cut = 7.5 / 128
        box.n_crit = 192
    return box


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling every 100 ms and wait (up to 3 s) for the first sample."""
        self.first = 0
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self):
        """The timed region starts: later summaries use samples from here on."""
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)                      # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines[self.first:]:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (N > 1: one independent replica per rank)
# ---------------------------------------------------------------------------
def max_over_ranks(values, device=None):
    """Element-wise maximum of `values` over all ranks of the default process
    group (the values themselves when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def sum_over_ranks(values, device=None):
    """Element-wise sum of `values` over all ranks of the default process
    group (the values themselves when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def whole_job_rate(world, units_per_step, steps, total_ms):
    """Units all ranks processed per second over the slowest rank's time:
    every rank runs the same fixed per-rank workload (weak scaling)."""
    return world * units_per_step * steps / (total_ms * 1e-3)


# ---------------------------------------------------------------------------
# the reference arm: the CPU FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample_rate(box, w, target_fraction=0.03, steps=1, warmup=0, report=None, xi_softened=False,
                       rsqrt_refined=False):
    """Time the oracle: build + lists once, then `steps` samples of forward +
    adjoint over a contiguous range of groups holding ~target_fraction of the
    interactions.  Each step is charged its share of the build + lists time."""
    import oracle
    t0 = time.perf_counter()
    ot = oracle.OracleTree(box.pos, box.mass, box.n_leaf, box.n_crit)
    ot.lists(box.r_cut, box.theta)
    t_build = time.perf_counter() - t0
    ex = ot.export()
    inter = ex.gcount * np.diff(ex.loff)
    total = int(inter.sum())
    cum = np.cumsum(inter)
    g1 = int(np.searchsorted(cum, target_fraction * total)) + 1
    sample = int(cum[g1 - 1])
    frac = sample / total
    w64 = w.astype(np.float64)
    times = []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        ot.list_forces_range(0, g1, box.G, box.eps, box.r_cut, xi_softened=xi_softened, rsqrt_refined=rsqrt_refined)
        ot.list_vjp_range(0, g1, box.G, box.eps, box.r_cut, w64, xi_softened=xi_softened,
                          rsqrt_refined=rsqrt_refined)
        dt = time.perf_counter() - t0 + frac * t_build
        if s >= warmup:
            times.append(dt)
    cores = oracle.num_threads()
    per_step = 2 * sample
    return {"per_step_interactions": per_step, "times": times, "cores": cores,
            "sample": f"groups [0,{g1}) of {ex.gfirst.size}: {sample} of {total} pair "
                      f"interactions (x2 forward+adjoint); build+lists {t_build:.2f}s charged "
                      f"pro rata ({frac:.3f})", "frac": frac, "t_build": t_build}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1211_4406_gb300 import inputs
    box = inputs.config_box(CONFIG_K)
    w = inputs.cotangent(box.n, box.seed + 7)
    r = oracle_sample_rate(box, w, steps=args.steps, warmup=args.warmup,
                           xi_softened=getattr(args, "xi", "plain") == "softened",
                           rsqrt_refined=getattr(args, "rsqrt", "hardware") == "refined")
    total_t = sum(r["times"])
    value = r["per_step_interactions"] * len(r["times"]) / total_t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(r["times"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(workload_config(), **({} if getattr(args, "xi", "plain") == "plain" else
                                                 {"xi": "softened: cutoff argument 2 sqrt(r^2+eps^2)/r_cut"})),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_paper_regime(args, rank, world, local_rank):
    run_ours(args, rank, world, local_rank, paper_regime=True)


def run_ours(args, rank, world, local_rank, paper_regime=False):
    import torch

    from paper_1211_4406_gb300 import autotune
    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import CapturedStep, Params, ShortRangeTree, launch_count, measure_peak
    from paper_1211_4406_gb300.profile_step import traffic_for

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    box = bench_box(paper_regime)
    w = inputs.cotangent(box.n, box.seed + 7)
    pos_h = torch.tensor(box.pos).pin_memory()
    mass_h = torch.tensor(box.mass).pin_memory()
    cot_h = torch.tensor(w).pin_memory()
    pos = pos_h.to(dev)
    mass = mass_h.to(dev)
    cot = cot_h.to(dev)
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32", xi=args.xi,
                 rsqrt=args.rsqrt)
    tree = ShortRangeTree(pos, mass, prm)                   # allocating build (setup)
    st = tree.stats()
    wl = workload_config(paper_regime)["workload"]
    xkey = ("" if args.xi == "plain" else "|xi-softened") + ("" if args.rsqrt == "hardware" else "|rsqrt-refined")
    tile = autotune.tune_tile(tree, pos, mass, cot, key=f"{wl}|n{box.n}{xkey}")   # setup, not timed
    acc = torch.empty((box.n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((box.n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)

    # One step: rebuild the tree from the positions, then the forces and their
    # adjoint for the step's cotangent (known in advance: the loss is linear in
    # the accelerations) in one pass over the lists.
    def step(p, m, c, evs=None):
        if evs:
            evs[0].record(stream)
        tree.rebuild(p, m)
        if evs:
            evs[1].record(stream)
        tree.force_vjp(c, acc, grad)
        if evs:
            evs[2].record(stream)

    # The same step with the force and the adjoint as separate calls.
    def step_separate(evs):
        evs[0].record(stream)
        tree.rebuild(pos, mass)
        evs[1].record(stream)
        tree.force(acc)
        evs[2].record(stream)
        tree.vjp(cot, grad)
        evs[3].record(stream)

    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    for _ in range(args.warmup):
        flush.zero_()
        step(pos, mass, cot)
    torch.cuda.synchronize()
    status = tree.status()
    if status != 0:
        raise RuntimeError(f"tree status {status} after warm-up")

    # ---- device-resident timed region -------------------------------------
    clocks.mark()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    # The step replayed from one CUDA graph (the library's batched-launch
    # path): the same kernels as the direct calls, without a host launch per
    # kernel.  Kernel timing is on during the capture, so every replay also
    # times the one-pass kernel (external event nodes).
    tree.set_kernel_timing(True)
    l0 = launch_count()
    graph_step = CapturedStep(tree, pos, mass, cot, acc, grad)    # warm-up body + captured body
    kernels_per_step = (launch_count() - l0) // 2
    for _ in range(args.warmup):
        flush.zero_()
        graph_step.replay()
    torch.cuda.synchronize()
    t_step, k_fused_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = ev(), ev()
        e0.record(stream)
        graph_step.replay()
        e1.record(stream)
        e1.synchronize()
        t_step.append(e0.elapsed_time(e1))
        k_fused_ms.append(tree.kernel_ms()[1])   # the one-pass kernel of this replay
    launches = kernels_per_step * args.steps
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    if tree.status() != 0:
        raise RuntimeError("tree status after the timed region")

    # ---- the same step as direct calls, with its phases ------------------------
    per = []
    for _ in range(args.steps):
        flush.zero_()
        evs = [ev() for _ in range(3)]
        step(pos, mass, cot, evs)
        per.append(evs)
    torch.cuda.synchronize()
    t_build = [e[0].elapsed_time(e[1]) for e in per]
    t_fused = [e[1].elapsed_time(e[2]) for e in per]
    t_direct = [e[0].elapsed_time(e[2]) for e in per]

    # ---- the separate calls, each kernel timed by its own events ---------------
    sep, k_pair_ms, k_vjp_ms = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        evs = [ev() for _ in range(4)]
        step_separate(evs)
        sep.append(evs)
        kf, kv = tree.kernel_ms()
        k_pair_ms.append(kf)
        k_vjp_ms.append(kv)
    tree.set_kernel_timing(False)
    torch.cuda.synchronize()

    # ---- end to end from host buffers ---------------------------------------
    acc_h = torch.empty((box.n, 3), dtype=torch.float32).pin_memory()
    grad_h = torch.empty((box.n, 3), dtype=torch.float64).pin_memory()

    def e2e_step():
        # host inputs into the tensors the graph reads, one replay, results back
        pos.copy_(pos_h, non_blocking=True)
        mass.copy_(mass_h, non_blocking=True)
        cot.copy_(cot_h, non_blocking=True)
        graph_step.replay()
        acc_h.copy_(acc, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = _timed_replays(e2e_step, args.steps, flush, stream)
    h2d = pos_h.numel() * 8 + mass_h.numel() * 8 + cot_h.numel() * 4
    d2h = acc_h.numel() * 4 + grad_h.numel() * 8

    # ---- plain FP64 GPU path (same lists), for the speedup --------------------
    tree64 = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit,
                                              box.n_leaf, "fp64", xi=args.xi))
    acc64 = torch.empty((box.n, 3), dtype=torch.float64, device=dev)
    tree64.force(acc64)
    torch.cuda.synchronize()
    f64_ms = _timed_replays(lambda: tree64.force(acc64), 2, flush, stream)
    tree64.close()

    # ---- max over ranks --------------------------------------------------------
    inter = int(st["n_interactions"])
    per_step_inter = 2 * inter
    tot_ms, tot_e2e = max_over_ranks([sum(t_step), sum(e2e_ms)], device=dev)
    value = whole_job_rate(world, per_step_inter, args.steps, tot_ms)
    e2e_value = whole_job_rate(world, per_step_inter, args.steps, tot_e2e)

    if rank != 0:
        tree.close()
        return
    mean = lambda xs: sum(xs) / len(xs)
    sep_step = mean([e[0].elapsed_time(e[3]) for e in sep])
    fp32_pk, peak_basis = fp32_peak(dev, clk)
    # every group of this workload takes the packed kernels (none spans half
    # the box and eps > 0), so each launch processes all interactions

    def roofline(kernel, ms, flops, note):
        ach = flops * inter / (ms * 1e-3)
        return {"bound": "alu", "achieved": ach / 1e12, "peak": fp32_pk / 1e12, "unit": "TFLOP/s",
                "frac": ach / fp32_pk,
                "traffic": traffic_for(kernel, st["n_entries"]) if wl == "clustered-2M" else None,
                "traffic_basis": "ncu DRAM bytes of a 2^19-particle box of the same recipe, scaled by list entries",
                "kernel": f"{kernel} ({note})",
                "ms_per_launch": ms, "flops_per_interaction": flops, "peak_basis": peak_basis}

    kp_ms, kv_ms, kw_ms = mean(k_pair_ms), mean(k_vjp_ms), mean(k_fused_ms)
    soft = "true" if args.xi == "softened" else "false"
    rf = "true" if args.rsqrt == "refined" else "false"
    # the adjoint kernels of the tuned shape: E entries per thread; at E = 8 the
    # entry-packed kernel (four pairs of entries per thread) in the one pass and
    # four entries per thread for the adjoint alone
    adj_kernel = (lambda fwd: f"k_vjp_epack<4, {fwd}, {soft}, {rf}>" if fwd == "true" else
                  f"k_vjp_fused<4, {fwd}, {soft}, {rf}>") if tile[1] == 8 else \
        (lambda fwd: f"k_vjp_fused<{tile[1]}, {fwd}, {soft}, {rf}>")
    meas_ffma = measure_peak("fp32")
    meas_ffma2 = measure_peak("fp32x2")
    meas_dfma = measure_peak("fp64")
    line = {
        "metric": METRIC.replace("clustered 2M box", "clustered 2M box, paper's list regime") if paper_regime
        else METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(paper_regime), tile_autotuned={"forward_particles_per_thread": tile[0],
                                                          "adjoint_entries_per_thread": tile[1]},
                       **({} if args.xi == "plain" else {"xi": "softened: cutoff argument 2 sqrt(r^2+eps^2)/r_cut"}),
                       **({} if args.rsqrt == "hardware" else
                          {"rsqrt": "refined: 1/s from an estimate and the paper's third-order step"})),
        "roofline": roofline(adj_kernel("true"), kw_ms, FUSED_FLOPS_PER_INTERACTION,
                             "one pass: forward (Eq. 2 x Eq. 3) and adjoint; the largest share of the step"),
        "roofline_forward": roofline(f"k_pair_packed<{tile[0]}, 8, {soft}, {rf}>", kp_ms, FLOPS_PER_INTERACTION,
                                     "FP32 forward pair kernel, separate call"),
        "roofline_adjoint": roofline(adj_kernel("false"), kv_ms,
                                     VJP_FLOPS_PER_INTERACTION, "FP32 adjoint pair kernel, separate call"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": tot_e2e / args.steps},
        "gpu_launches": launches,
        "gpu_launches_basis": f"{kernels_per_step} kernels per graph replay x {args.steps} replays",
        "step": "one CUDA-graph replay (CapturedStep) of tp_rebuild_tree + tp_short_range_force_vjp",
        "clocks": clk,
        "direct_calls": {"ms_per_step": mean(t_direct), "value": per_step_inter / (mean(t_direct) * 1e-3)},
        "phases_ms": {"build": mean(t_build), "force_and_vjp_one_pass": mean(t_fused),
                      "force_fp32_separate": mean([e[1].elapsed_time(e[2]) for e in sep]),
                      "vjp_fp32_separate": mean([e[2].elapsed_time(e[3]) for e in sep]),
                      "force_fp64": mean(f64_ms)},
        "separate_calls": {"ms_per_step": sep_step, "value": per_step_inter / (sep_step * 1e-3)},
        "forward_interactions_per_s": inter / (kp_ms * 1e-3),
        "adjoint_interactions_per_s": inter / (kv_ms * 1e-3),
        "fp64_forward_interactions_per_s": inter / (mean(f64_ms) * 1e-3),
        "fp32_over_fp64_forward_speedup": mean(f64_ms) / kp_ms,
        "forward_paper_convention_frac": PAPER_FLOPS_PER_INTERACTION * inter / (kp_ms * 1e-3) / fp32_pk,
        "measured_peaks_tflops": {"ffma": meas_ffma / 1e12, "ffma2": meas_ffma2 / 1e12,
                                  "dfma": meas_dfma / 1e12},
        "tree": {k: st[k] for k in ("n_nodes", "n_groups", "n_entries", "n_interactions", "n_useful",
                                    "n_ambiguous", "mean_ni", "mean_nj", "max_nj")},
        "useful_fraction": st["n_useful"] / max(1, st["n_interactions"]),
        "useful_fraction_basis": "pairs with a non-zero Eq. 2 term (0 < r < r_cut, decided in FP64) among "
                                 "the sum over groups of n_i * n_j that value counts",
    }
    tree.close()
    if not paper_regime and args.xi == "plain" and args.rsqrt == "hardware" and not args.no_sub_records:
        # the other configurations, each measured briefly after the timed
        # region above with its own clock sample and kernel count
        subs = {}
        for name, fn in (("uniform-32k", sub_uniform_32k), ("batched-64", sub_batched_64),
                         ("clustered-134M", sub_clustered_134m)):
            if name == "clustered-134M" and args.no_c5:
                continue
            try:
                subs[name] = fn(dev, stream, flush, local_rank)
            except Exception as e:              # a sub-record never voids the main line
                subs[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.synchronize()
        line["sub_records"] = subs
    if world == 1 and not args.no_cpu_baseline and not paper_regime:
        r = oracle_sample_rate(box, w, steps=1, xi_softened=args.xi == "softened",
                               rsqrt_refined=args.rsqrt == "refined")
        line["cpu_baseline"] = {"value": r["per_step_interactions"] / r["times"][0], "unit": UNIT,
                                "cores": r["cores"], "kind": "oracle", "sample": r["sample"]}
    print(json.dumps(line), flush=True)


def _sampled(clock_gpu, fn):
    """fn() with nvidia-smi sampling around it: (fn's result, clock summary)."""
    clocks = ClockSampler(clock_gpu)
    clocks.start()
    clocks.mark()
    try:
        out = fn()
    finally:
        clk = clocks.stop()
    return out, clk


def sub_uniform_32k(dev, stream, flush, local_rank, steps=10, warmup=3):
    """C1: the plain FP64 path on the uniform 32^3 box, rebuild + force +
    adjoint per step (device-timed, L2 flushed), with the FP32 step beside it."""
    import torch

    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, ShortRangeTree, launch_count
    box = inputs.config_box(1)
    pos, mass = torch.tensor(box.pos, device=dev), torch.tensor(box.mass, device=dev)
    cot64 = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device=dev).double()
    out = {"config": "N = 32^3 uniform, r_cut = 3/32, eps = 1/1600, theta = 0.5, n_crit = 64"}
    for prec, adt in (("fp64", torch.float64), ("fp32", torch.float32)):
        tree = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, prec))
        acc = torch.empty((box.n, 3), dtype=adt, device=dev)
        grad = torch.empty((box.n, 3), dtype=torch.float64, device=dev)
        cot = cot64.to(adt)

        def step():
            tree.rebuild(pos, mass)
            tree.force(acc)
            tree.vjp(cot, grad)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        l0 = launch_count()
        ms, clk = _sampled(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0,
                           lambda: _timed_replays(step, steps, flush, stream))
        inter = int(tree.stats()["n_interactions"])
        if tree.status() != 0:
            raise RuntimeError(f"{prec} tree status {tree.status()}")
        tree.close()
        m = sum(ms) / len(ms)
        out[prec] = {"ms_per_step": m, "interactions_per_s": 2 * inter / (m * 1e-3),
                     "gpu_launches_per_step": (launch_count() - l0) // steps, "clocks": clk}
        out["n_interactions"] = inter
    out["fp32_over_fp64_step_speedup"] = out["fp64"]["ms_per_step"] / out["fp32"]["ms_per_step"]
    return out


def sub_batched_64(dev, stream, flush, local_rank, steps=5, warmup=3):
    """C3: the 64 batched boxes (autotuned n_crit and tile), rebuild plus
    forces and adjoint of every box as one CUDA-graph replay."""
    import torch

    from paper_1211_4406_gb300 import autotune, inputs
    from paper_1211_4406_gb300.api import CapturedStep, Params, ShortRangeTree, launch_count
    t0 = time.perf_counter()
    boxes = inputs.batched_boxes(64)
    kinds = ["uniform" if b % 2 == 0 else "clustered" for b in range(64)]
    base = [Params(b.G, b.eps, b.r_cut, b.theta, 64, 8, "fp32") for b in boxes]
    ncrit = autotune.tune_boxes(boxes, kinds, base, reps=2)
    prm = [Params(b.G, b.eps, b.r_cut, b.theta, c, 8, "fp32") for b, c in zip(boxes, ncrit)]
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    pos = torch.tensor(np.concatenate([b.pos for b in boxes]), device=dev)
    mass = torch.tensor(np.concatenate([b.mass for b in boxes]), device=dev)
    cot = torch.tensor(np.concatenate([inputs.cotangent(b.n, b.seed + 7) for b in boxes]), device=dev)
    tree = ShortRangeTree(pos, mass, prm, box_offsets=offs.tolist())
    tile = autotune.tune_tile(tree, pos, mass, cot, key=f"batched-64|n{tree.n}")
    acc = torch.empty((tree.n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((tree.n, 3), dtype=torch.float64, device=dev)
    l0 = launch_count()
    step = CapturedStep(tree, pos, mass, cot, acc, grad)
    per_replay = (launch_count() - l0) // 2
    setup = time.perf_counter() - t0
    for _ in range(warmup):
        step.replay()
    torch.cuda.synchronize()
    ms, clk = _sampled(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0,
                       lambda: _timed_replays(step.replay, steps, flush, stream))
    st = tree.stats()
    if tree.status() != 0:
        raise RuntimeError("batched tree status")
    tree.close()
    m = sum(ms) / len(ms)
    return {"config": "64 boxes, N_b log-uniform in [16^3, 96^3], even uniform, odd clustered, "
                      "r_cut = 3/N_b^(1/3), theta = 0.5, one CUDA-graph replay per step",
            "n_total": int(tree.n), "n_interactions": int(st["n_interactions"]),
            "ms_per_step": m, "interactions_per_s": 2 * st["n_interactions"] / (m * 1e-3),
            "useful_fraction": st["n_useful"] / max(1, st["n_interactions"]),
            "tile_autotuned": list(tile), "gpu_launches_per_step": per_replay, "setup_s": setup, "clocks": clk}


def sub_clustered_134m(dev, stream, flush, local_rank, steps=1, warmup=1):
    """C5: the 512^3 clustered box (chunked lists), rebuild plus forces and
    adjoint in one pass per step."""
    import torch

    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, ShortRangeTree, launch_count
    t0 = time.perf_counter()
    box = inputs.config_box(5)
    t_gen = time.perf_counter() - t0
    n = box.n
    pos, mass = torch.from_numpy(box.pos).to(dev), torch.from_numpy(box.mass).to(dev)
    cot = torch.from_numpy(inputs.cotangent(n, box.seed + 7)).to(dev)
    tree = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32"))
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((n, 3), dtype=torch.float64, device=dev)

    def step():
        tree.rebuild(pos, mass)
        tree.force_vjp(cot, acc, grad)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    l0 = launch_count()
    ms, clk = _sampled(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0,
                       lambda: _timed_replays(step, steps, flush, stream))
    launches = (launch_count() - l0) // steps
    st = tree.stats()
    if tree.status() != 0:
        raise RuntimeError("134M tree status")
    tree.close()
    m = sum(ms) / len(ms)
    return {"config": "N = 512^3 clustered (10^5 halos), r_cut = 3/512, eps = 1/25600, theta = 0.5, chunked lists",
            "n_interactions": int(st["n_interactions"]), "n_windows": int(st["n_windows"]),
            "ms_per_step": m, "interactions_per_s": 2 * st["n_interactions"] / (m * 1e-3),
            "gpu_launches_per_step": launches, "generate_inputs_s": t_gen, "clocks": clk}


def _timed_replays(fn, steps, flush, stream):
    """Per-call device times (ms) of fn() over `steps` calls, L2 flushed before each."""
    import torch
    out = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def run_batched(args, rank, world, local_rank):
    """64 independent periodic boxes (sizes log-uniform in [16^3, 96^3], even
    boxes uniform, odd boxes clustered), n_crit per box from the autotuner, the
    whole step (rebuild + FP32 force + FP32 adjoint of every box) captured in
    one CUDA graph and timed as one replay.  With N ranks the 64 boxes are
    shared among them (strong scaling: the same 64 boxes at every N)."""
    import torch

    from paper_1211_4406_gb300 import autotune
    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import CapturedStep, Params, ShortRangeTree, launch_count

    from paper_1211_4406_gb300.domain import partition_boxes

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    all_boxes = inputs.batched_boxes(64)
    all_kinds = ["uniform" if b % 2 == 0 else "clustered" for b in range(64)]
    base = [Params(b.G, b.eps, b.r_cut, b.theta, 64, 8, "fp32") for b in all_boxes]
    t0 = time.perf_counter()
    ncrit_all = autotune.tune_boxes(all_boxes, all_kinds, base, reps=2)
    t_tune = time.perf_counter() - t0
    # with several ranks, each takes a share of the independent boxes (no
    # collective on the data path): longest-processing-time split by each
    # box's interaction count, the same on every rank
    if world > 1:
        costs = []
        for b, c in zip(all_boxes, ncrit_all):
            tb = ShortRangeTree(torch.tensor(b.pos, device=dev), torch.tensor(b.mass, device=dev),
                                Params(b.G, b.eps, b.r_cut, b.theta, c, 8, "fp32"))
            costs.append(tb.stats()["n_interactions"])
            tb.close()
        mine = partition_boxes(costs, world)[rank]
    else:
        mine = list(range(64))
    boxes = [all_boxes[b] for b in mine]
    ncrit = [ncrit_all[b] for b in mine]
    prm = [Params(b.G, b.eps, b.r_cut, b.theta, c, 8, "fp32") for b, c in zip(boxes, ncrit)]
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    pos_h = torch.tensor(np.concatenate([b.pos for b in boxes])).pin_memory()
    mass_h = torch.tensor(np.concatenate([b.mass for b in boxes])).pin_memory()
    cot_h = torch.tensor(np.concatenate([inputs.cotangent(b.n, b.seed + 7) for b in boxes])).pin_memory()
    pos, mass, cot = pos_h.to(dev), mass_h.to(dev), cot_h.to(dev)
    tree = ShortRangeTree(pos, mass, prm, box_offsets=offs.tolist())
    st = tree.stats()
    n = tree.n
    tile = autotune.tune_tile(tree, pos, mass, cot, key=f"batched-64|n{n}")
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((n, 3), dtype=torch.float64, device=dev)
    l0 = launch_count()
    step = CapturedStep(tree, pos, mass, cot, acc, grad)      # warm-up body + captured body
    per_replay = (launch_count() - l0) // 2
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step.replay()
    torch.cuda.synchronize()
    if tree.status() != 0:
        raise RuntimeError("tree status after warm-up replays")
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    clocks.mark()
    ms = _timed_replays(step.replay, args.steps, flush, stream)
    clk = clocks.stop()
    if tree.status() != 0:
        raise RuntimeError("tree status after the timed replays")
    acc_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    grad_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()

    def e2e():
        pos.copy_(pos_h, non_blocking=True)
        mass.copy_(mass_h, non_blocking=True)
        cot.copy_(cot_h, non_blocking=True)
        step.replay()
        acc_h.copy_(acc, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)

    e2e_ms = _timed_replays(e2e, args.steps, flush, stream)
    inter = int(st["n_interactions"])
    tot_ms, tot_e2e = max_over_ranks([sum(ms), sum(e2e_ms)], device=dev)
    inter_all = int(sum_over_ranks([inter], device=dev)[0])        # each rank has its own share of boxes
    value = 2 * inter_all * args.steps / (tot_ms * 1e-3)
    e2e_value = 2 * inter_all * args.steps / (tot_e2e * 1e-3)
    n_all = int(sum_over_ranks([n], device=dev)[0])
    tree.close()
    if rank != 0:
        return
    hist = {}
    for c in ncrit:
        hist[str(c)] = hist.get(str(c), 0) + 1
    line = {
        "metric": METRIC.replace("clustered 2M box", "64 batched boxes"), "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched-64", "nbox": 64, "n_total": n_all,
                   "n_min": int(min(b.n for b in all_boxes)), "n_max": int(max(b.n for b in all_boxes)),
                   "kinds": "even uniform, odd clustered",
                   "sharding": "one rank" if world == 1 else
                   f"{world} ranks, boxes split by interaction count (LPT), rank 0 has {len(mine)} boxes",
                   "r_cut": "3/N_b^(1/3)", "eps": "1/(50 N_b^(1/3))", "theta": 0.5,
                   "n_crit_autotuned": hist,
                   "tile_autotuned": {"forward_particles_per_thread": tile[0], "adjoint_entries_per_thread": tile[1]},
                   "graph": "rebuild + one-pass forces and adjoint of all boxes in one replay",
                   "l2": "flushed (256 MiB write) before every timed replay"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": pos_h.numel() * 8 + mass_h.numel() * 8
                + cot_h.numel() * 4, "d2h_bytes_per_step": acc_h.numel() * 4 + grad_h.numel() * 8,
                "ms_per_step": tot_e2e / args.steps},
        "gpu_launches": per_replay * args.steps, "clocks": clk,
        "autotune_s": t_tune,
        "tree": {k: st[k] for k in ("n_nodes", "n_groups", "n_entries", "n_interactions", "n_useful", "mean_ni",
                                    "mean_nj", "max_nj", "nbox")},
        "useful_fraction": st["n_useful"] / max(1, st["n_interactions"]),
    }
    print(json.dumps(line), flush=True)


def run_uniform_fp64(args, rank, world, local_rank):
    """The plain FP64 path (FP64 pair arithmetic, same tree and lists) on the
    uniform 32^3 box: rebuild + FP64 force + FP64 adjoint per step, with the
    FP32 path's step time on the same box beside it."""
    import torch

    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, ShortRangeTree, launch_count

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    box = inputs.config_box(1)
    pos_h = torch.tensor(box.pos).pin_memory()
    mass_h = torch.tensor(box.mass).pin_memory()
    cot_h = torch.tensor(inputs.cotangent(box.n, box.seed + 7)).pin_memory()
    pos, mass = pos_h.to(dev), mass_h.to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for prec, adt in (("fp64", torch.float64), ("fp32", torch.float32)):
        tree = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit,
                                                box.n_leaf, prec))
        cot = cot_h.to(dev).to(adt)
        acc = torch.empty((box.n, 3), dtype=adt, device=dev)
        grad = torch.empty((box.n, 3), dtype=torch.float64, device=dev)

        def step():
            tree.rebuild(pos, mass)
            tree.force(acc)
            tree.vjp(cot, grad)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        l0 = launch_count()
        ms = _timed_replays(step, args.steps, flush, stream)
        res[prec] = {"ms": ms, "launches": launch_count() - l0, "stats": tree.stats(),
                     "status": tree.status()}
        if prec == "fp64":
            def e2e():
                pos.copy_(pos_h, non_blocking=True)
                mass.copy_(mass_h, non_blocking=True)
                cot.copy_(cot_h.to(adt), non_blocking=True)
                step()
                acc.cpu()
                grad.cpu()
            res["e2e_ms"] = _timed_replays(e2e, args.steps, flush, stream)
        tree.close()
        if res[prec]["status"] != 0:
            raise RuntimeError(f"{prec} tree status {res[prec]['status']}")
    inter = int(res["fp64"]["stats"]["n_interactions"])
    tot_ms, tot_e2e = max_over_ranks([sum(res["fp64"]["ms"]), sum(res["e2e_ms"])], device=dev)
    value = whole_job_rate(world, 2 * inter, args.steps, tot_ms)
    if rank != 0:
        return
    st = res["fp64"]["stats"]
    fp32_ms = sum(res["fp32"]["ms"]) / args.steps
    line = {
        "metric": "short-range interactions/s (plain FP64 forward + adjoint, uniform 32^3 box)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "uniform-32k", "n": box.n, "r_cut": "3/32", "eps": "1/1600", "theta": 0.5,
                   "n_crit": box.n_crit, "n_leaf": box.n_leaf, "seed": box.seed,
                   "l2": "flushed (256 MiB write) before every timed step"},
        "e2e": {"value": whole_job_rate(world, 2 * inter, args.steps, tot_e2e), "unit": UNIT,
                "h2d_bytes_per_step": box.n * (24 + 8 + 24), "d2h_bytes_per_step": box.n * (24 + 24),
                "ms_per_step": tot_e2e / args.steps},
        "gpu_launches": res["fp64"]["launches"],
        "fp32_step_ms": fp32_ms, "fp32_over_fp64_step_speedup": (tot_ms / args.steps) / fp32_ms,
        "tree": {k: st[k] for k in ("n_nodes", "n_groups", "n_entries", "n_interactions", "n_useful", "mean_ni",
                                    "mean_nj", "max_nj")},
        "useful_fraction": st["n_useful"] / max(1, st["n_interactions"]),
    }
    print(json.dumps(line), flush=True)


def run_large(args, rank, world, local_rank):
    """The throughput workload at the paper's per-node load: N = 512^3
    clustered particles (10^5 NFW halos), r_cut = 3/512, eps = 1/25600,
    theta = 0.5, FP32 forward + adjoint in one pass.  Its lists (~1.4e10
    entries) do not fit in device memory, so the tree runs in chunked mode
    (windows of groups with bounded list memory, planned once per step, each
    walked once for both the forces and the adjoint)."""
    import torch

    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, ShortRangeTree, launch_count

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    box = inputs.config_box(5)
    w = inputs.cotangent(box.n, box.seed + 7)
    t_gen = time.perf_counter() - t0
    pos_h = torch.from_numpy(box.pos).pin_memory()
    mass_h = torch.from_numpy(box.mass).pin_memory()
    cot_h = torch.from_numpy(w).pin_memory()
    pos, mass, cot = pos_h.to(dev), mass_h.to(dev), cot_h.to(dev)
    t0 = time.perf_counter()
    tree = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf,
                                            "fp32"))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    st = tree.stats()
    acc = torch.empty((box.n, 3), dtype=torch.float32, device=dev)
    grad = torch.empty((box.n, 3), dtype=torch.float64, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        tree.rebuild(pos, mass)
        tree.force_vjp(cot, acc, grad)
    torch.cuda.synchronize()
    if tree.status() != 0:
        raise RuntimeError(f"tree status {tree.status()} after warm-up")
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    clocks.mark()
    l0 = launch_count()
    phases = []
    for _ in range(args.steps):
        e = [ev() for _ in range(3)]
        e[0].record(stream)
        tree.rebuild(pos, mass)
        e[1].record(stream)
        tree.force_vjp(cot, acc, grad)          # each window walked once for both
        e[2].record(stream)
        e[2].synchronize()
        phases.append([e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])])
    launches = launch_count() - l0
    clk = clocks.stop()
    if tree.status() != 0:
        raise RuntimeError("tree status after the timed steps")
    st = tree.stats()
    acc_h = torch.empty((box.n, 3), dtype=torch.float32).pin_memory()
    grad_h = torch.empty((box.n, 3), dtype=torch.float64).pin_memory()

    def e2e():
        pos.copy_(pos_h, non_blocking=True)
        mass.copy_(mass_h, non_blocking=True)
        cot.copy_(cot_h, non_blocking=True)
        tree.rebuild(pos, mass)
        tree.force_vjp(cot, acc, grad)
        acc_h.copy_(acc, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    e2e_ms = _timed_replays(e2e, 1, flush, stream)
    inter = int(st["n_interactions"])
    step_ms = [sum(p) for p in phases]
    tot_ms, tot_e2e = max_over_ranks([sum(step_ms), sum(e2e_ms) * args.steps], device=dev)
    value = whole_job_rate(world, 2 * inter, args.steps, tot_ms)
    tree.close()
    if rank != 0:
        return
    mean = lambda i: sum(p[i] for p in phases) / len(phases)
    line = {
        "metric": METRIC.replace("clustered 2M box", "clustered 134M box"), "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "clustered-134M", "n": box.n, "halos": 100000, "r_cut": "3/512",
                   "eps": "1/25600", "theta": 0.5, "n_crit": box.n_crit, "n_leaf": box.n_leaf, "seed": box.seed,
                   "lists": f"chunked: {st['n_windows']} windows of groups",
                   "l2": "inputs (4.3 GB of positions and masses) larger than L2"},
        "e2e": {"value": whole_job_rate(world, 2 * inter, args.steps, tot_e2e), "unit": UNIT,
                "h2d_bytes_per_step": box.n * (24 + 8 + 12), "d2h_bytes_per_step": box.n * (12 + 24),
                "ms_per_step": tot_e2e / args.steps},
        "gpu_launches": launches, "clocks": clk,
        "phases_ms": {"build": mean(0), "force_and_vjp_one_pass": mean(1)},
        "setup_s": {"generate_inputs": t_gen, "allocating_build": t_build},
        "tree": {k: st[k] for k in ("n_nodes", "n_groups", "n_entries", "n_interactions", "mean_ni",
                                    "mean_nj", "max_nj", "n_windows")},
    }
    print(json.dumps(line), flush=True)


def run_leapfrog(args, rank, world, local_rank):
    """The adjoint workload: the gradient of L = sum w . a_T with respect to
    x0 through 10 FP32 kick-drift-kick steps (dt = 1e-3) on the clustered
    262k box (250 halos, r_cut = 3/64, eps = 1/3200), with one checkpoint per
    step: 11 force evaluations forward, 10 rebuilds + adjoints and the first
    force's adjoint backward.  Trees are rebuilt in place across the steps."""
    import torch

    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, ShortRangeTree, launch_count
    from paper_1211_4406_gb300.autograd import leapfrog

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    box = inputs.config_box(4)
    steps, dt = 10, 1e-3
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32")
    pos_h = torch.tensor(box.pos).pin_memory()
    w_h = torch.tensor(inputs.cotangent(box.n, box.seed + 7)).pin_memory()
    mass = torch.tensor(box.mass, device=dev)
    wt = w_h.to(dev).double()
    x0 = pos_h.to(dev).requires_grad_(True)
    v0 = torch.zeros_like(x0)
    t0 = ShortRangeTree(x0.detach(), mass, prm)
    inter = int(t0.stats()["n_interactions"])
    t0.close()

    def grad_once(reuse=True):
        x0.grad = None
        _, _, aT = leapfrog(x0, v0, mass, prm, dt, steps, reuse_trees=reuse)
        (aT.double() * wt).sum().backward()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        grad_once()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    clocks.mark()
    l0 = launch_count()
    ms = _timed_replays(grad_once, args.steps, flush, stream)
    launches = launch_count() - l0
    clk = clocks.stop()
    ms_fresh = _timed_replays(lambda: grad_once(False), max(2, args.steps // 4), flush, stream)
    g = x0.grad.detach()
    e2e_ms = _timed_replays(lambda: (x0.data.copy_(pos_h, non_blocking=True), grad_once(),
                                     g.cpu()), max(2, args.steps // 4), flush, stream)
    per = 2 * (steps + 1) * inter              # forces and adjoints of one gradient
    tot_ms, = max_over_ranks([sum(ms)], device=dev)
    value = whole_job_rate(world, per, args.steps, tot_ms)
    if rank != 0:
        return
    line = {
        "metric": "short-range interactions/s (FP32 10-step leapfrog gradient, clustered 262k box)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "leapfrog-262k", "n": box.n, "halos": 250, "r_cut": "3/64", "eps": "1/3200",
                   "theta": 0.5, "n_crit": box.n_crit, "kdk_steps": steps, "dt": dt,
                   "step": "one gradient: 11 forces forward, 11 adjoints backward, checkpoint per KDK step",
                   "l2": "flushed (256 MiB write) before every timed gradient"},
        "e2e": {"value": whole_job_rate(world, per, len(e2e_ms), sum(e2e_ms)), "unit": UNIT,
                "h2d_bytes_per_step": box.n * 24, "d2h_bytes_per_step": box.n * 24,
                "ms_per_step": sum(e2e_ms) / len(e2e_ms)},
        "gpu_launches": launches, "clocks": clk,
        "interactions_per_force": inter,
        "ms_per_gradient_fresh_trees": sum(ms_fresh) / len(ms_fresh),
    }
    print(json.dumps(line), flush=True)


def run_treepm(args, rank, world, local_rank):
    """The whole TreePM acceleration of the clustered 2M box: rebuild the
    tree, the FP32 short-range force (Eq. 2 with Eq. 3, r_cut = 3/128), and
    the long-range PM force on the 128^3 mesh (three mesh spacings per r_cut,
    as the paper sets it) added onto it."""
    import torch

    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import CapturedStep, Params, PMSolver, ShortRangeTree, launch_count

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    box = inputs.config_box(CONFIG_K)
    n_mesh = 128
    pos_h = torch.tensor(box.pos).pin_memory()
    pos = pos_h.to(dev)
    mass = torch.tensor(box.mass, device=dev)
    tree = ShortRangeTree(pos, mass, Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32"))
    pm = PMSolver(n_mesh, box.r_cut, box.G)
    acc = torch.empty((box.n, 3), dtype=torch.float32, device=dev)
    acc_h = torch.empty((box.n, 3), dtype=torch.float32).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    phases = []

    def step(record=False):
        e = [ev() for _ in range(4)] if record else None
        if record:
            e[0].record(stream)
        tree.rebuild(pos, mass)
        if record:
            e[1].record(stream)
        tree.force(acc)
        if record:
            e[2].record(stream)
        pm.force(pos, mass, out=acc, accumulate=True)
        if record:
            e[3].record(stream)
            phases.append(e)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the whole step (rebuild, short-range force, PM force added) as one graph replay
    l0 = launch_count()
    graph_step = CapturedStep(tree, pos, mass, None, acc, None, with_vjp=False, pm=pm)
    kernels_per_step = (launch_count() - l0) // 2
    for _ in range(args.warmup):
        graph_step.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    clocks.mark()
    ms = _timed_replays(graph_step.replay, args.steps, flush, stream)
    launches = kernels_per_step * args.steps
    clk = clocks.stop()
    direct = _timed_replays(lambda: step(True), args.steps, flush, stream)      # phases, direct calls
    pm_only = _timed_replays(lambda: pm.force(pos, mass, out=acc), args.steps, flush, stream)
    e2e_ms = _timed_replays(lambda: (pos.copy_(pos_h, non_blocking=True), graph_step.replay(),
                                     acc_h.copy_(acc, non_blocking=True)), max(2, args.steps // 2), flush, stream)
    tot_ms, tot_e2e = max_over_ranks([sum(ms), sum(e2e_ms)], device=dev)
    value = whole_job_rate(world, box.n, args.steps, tot_ms)
    st = tree.stats()
    if rank != 0:
        return
    mean = lambda xs: sum(xs) / len(xs)
    ph = {"build": mean([e[0].elapsed_time(e[1]) for e in phases]),
          "short_range_force": mean([e[1].elapsed_time(e[2]) for e in phases]),
          "pm_force": mean([e[2].elapsed_time(e[3]) for e in phases]),
          "pm_force_alone_l2_flushed": mean(pm_only)}
    fp32_pk, _ = fp32_peak(dev, clk)
    ach = FLOPS_PER_INTERACTION * st["n_interactions"] / (ph["short_range_force"] * 1e-3)
    line = {
        "metric": "particles/s (whole TreePM acceleration: rebuild + FP32 short-range + PM on 128^3, clustered 2M box)",
        "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "treepm-2M", "n": box.n, "halos": 2000, "r_cut": "3/128", "eps": "1/6400",
                   "theta": 0.5, "n_crit": box.n_crit, "n_mesh": n_mesh,
                   "l2": "flushed (256 MiB write) before every timed step"},
        "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": fp32_pk / 1e12, "unit": "TFLOP/s",
                     "frac": ach / fp32_pk, "traffic": None,
                     "kernel": "short-range force call (k_pair_packed + general kernel), the largest share",
                     "flops_per_interaction": FLOPS_PER_INTERACTION},
        "phases_ms": ph,
        "e2e": {"value": whole_job_rate(world, box.n, len(e2e_ms), tot_e2e), "unit": "particles/s",
                "h2d_bytes_per_step": box.n * 24, "d2h_bytes_per_step": box.n * 12,
                "ms_per_step": tot_e2e / len(e2e_ms)},
        "gpu_launches": launches,
        "gpu_launches_basis": f"{kernels_per_step} library kernels per graph replay (plus cuFFT's) x {args.steps} replays",
        "step": "one CUDA-graph replay (CapturedStep with the PM solver) of rebuild + short-range force + PM force",
        "direct_calls_ms_per_step": mean(direct),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    pm.close()
    tree.close()


def run_treepm_leapfrog(args, rank, world, local_rank):
    """Multiple-stepsize TreePM integration of the clustered 2M box (the
    paper's schedule: per step one PM cycle on the 128^3 mesh and two PP
    kick-drift-kick sub-steps of dt/2), timed per step; the second sub-step's
    tree rebuilt (as the paper does) or refitted from the first (lists kept)."""
    import torch

    from paper_1211_4406_gb300 import build as libbuild
    from paper_1211_4406_gb300 import inputs
    from paper_1211_4406_gb300.api import Params, PMSolver, launch_count
    from paper_1211_4406_gb300.autograd import treepm_leapfrog

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    box = inputs.config_box(CONFIG_K)
    dt = 1e-4
    prm = Params(box.G, box.eps, box.r_cut, box.theta, box.n_crit, box.n_leaf, "fp32")
    pm = PMSolver(128, box.r_cut, box.G)
    x0 = torch.tensor(box.pos, device=dev)
    v0 = torch.zeros_like(x0)
    mass = torch.tensor(box.mass, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    launches = 0
    clk = None
    for refit in (True, False):
        def steps(k):
            with torch.no_grad():
                treepm_leapfrog(x0, v0, mass, prm, pm, dt, k, refit=refit)
        for _ in range(args.warmup):
            steps(1)
        torch.cuda.synchronize()
        # time k steps and 1 step: their difference is k - 1 steps without the initial forces
        k = max(2, args.steps // 4)
        if refit:
            clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
            clocks.start()
            clocks.mark()
            l0 = launch_count()
        t_k = _timed_replays(lambda: steps(k), 3, flush, stream)
        t_1 = _timed_replays(lambda: steps(1), 3, flush, stream)
        if refit:
            launches = launch_count() - l0
            clk = clocks.stop()
        res[refit] = (sorted(t_k)[1] - sorted(t_1)[1]) / (k - 1)
    # one gradient through 3 steps (refitted second sub-steps): d(sum w . a_T)/dx0
    w = torch.tensor(inputs.cotangent(box.n, box.seed + 7), device=dev).double()
    xg = x0.clone().requires_grad_(True)

    def grad_once():
        xg.grad = None
        _, _, a_pp, a_pm = treepm_leapfrog(xg, v0, mass, prm, pm, dt, 3, refit=True)
        ((a_pp.double() + a_pm.double()) * w).sum().backward()

    grad_once()
    torch.cuda.synchronize()
    t_grad = sorted(_timed_replays(grad_once, 3, flush, stream))[1]
    ms_step, = max_over_ranks([res[True]], device=dev)
    if rank != 0:
        return
    line = {
        "metric": "particles x steps/s (multiple-stepsize TreePM integration, PM + 2 PP sub-steps per step, "
                  "clustered 2M box)",
        "value": world * box.n / (ms_step * 1e-3), "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "treepm-leapfrog-2M", "n": box.n, "r_cut": "3/128", "eps": "1/6400", "theta": 0.5,
                   "n_crit": box.n_crit, "n_mesh": 128, "dt": dt,
                   "step": "PM kick, 2 x (PP kick, drift, tree, PP force, PP kick), PM force, PM kick",
                   "second_sub_step": "refit (lists kept)",
                   "l2": "flushed (256 MiB write) before every timed run"},
        "ms_per_step_rebuild_both_sub_steps": res[False],
        "ms_per_step_refit_second_sub_step": res[True],
        "ms_per_gradient_3_steps": t_grad,
        "gradient": "d(sum w . (a_PP + a_PM)(x_T))/dx_0 through 3 steps, one checkpoint per step: 7 PP and 4 PM "
                    "forces forward; recomputation, 7 PP and 4 PM adjoints backward",
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    pm.close()


WORKLOADS = {"clustered-2M": run_ours, "batched-64": run_batched, "uniform-32k": run_uniform_fp64,
             "clustered-134M": run_large, "paper-regime-2M": run_paper_regime, "leapfrog-262k": run_leapfrog,
             "treepm-2M": run_treepm, "treepm-leapfrog-2M": run_treepm_leapfrog}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="leave out the default line's brief measurements of the other configurations")
    ap.add_argument("--no-c5", action="store_true",
                    help="leave the 512^3 box out of the default line's sub-records (its inputs take ~40 s to draw)")
    ap.add_argument("--workload", default="clustered-2M", choices=list(WORKLOADS),
                    help="clustered-2M (the default line); batched-64: 64 independent boxes, "
                         "autotuned n_crit, the whole step as one CUDA-graph replay; uniform-32k: "
                         "the plain FP64 path on the uniform 32^3 box; clustered-134M: "
                         "the 512^3 throughput box (chunked lists); paper-regime-2M: the 2M box with the "
                         "paper's list shapes (r_cut = 7.5 spacings, n_crit = 128); leapfrog-262k: the gradient "
                         "of a 10-step KDK chain (checkpointed adjoint); treepm-2M: the whole TreePM "
                         "acceleration (rebuild + short-range + PM on 128^3); treepm-leapfrog-2M: the "
                         "multiple-stepsize TreePM integrator (PM once, PP twice per step)")
    ap.add_argument("--rsqrt", default="hardware", choices=["hardware", "refined"],
                    help="1/s in the FP32 pair kernels for clustered-2M and paper-regime-2M: the hardware "
                         "reciprocal square root (default) or the paper's refinement of an estimate")
    ap.add_argument("--xi", default="plain", choices=["plain", "softened"],
                    help="cutoff argument of Eq. 3 for clustered-2M and paper-regime-2M: plain r (default) "
                         "or the softened sqrt(r^2+eps^2) of the paper's kernel")
    args = ap.parse_args()
    if args.xi != "plain" and args.workload not in ("clustered-2M", "paper-regime-2M"):
        ap.error(f"--xi {args.xi} applies to the clustered-2M and paper-regime-2M workloads only")
    if args.rsqrt != "hardware" and args.workload not in ("clustered-2M", "paper-regime-2M"):
        ap.error(f"--rsqrt {args.rsqrt} applies to the clustered-2M and paper-regime-2M workloads only")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload != "clustered-2M":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  f"the oracle arm is timed on the clustered-2M workload only"}))
            return
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        WORKLOADS[args.workload](args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
