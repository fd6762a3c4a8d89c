"""Host logic of the spatial decomposition (paper_1211_4406_gb300/domain.py) on
CPU: the multi-section cuts, their moving average and the cost-weighted sample
counts; and, with gloo ranks (world sizes 2 and 4), the whole exchange of one
step -- sampling, cuts, particle exchange, ghost exchange, per-domain forces
and adjoint, ghost gradients returned to their owners -- with the selections
and the per-domain sums taken by the oracle (the library's kernels need a
GPU; tests/test_gpu_domain.py checks them against the same oracle).  The
assembled forces equal the single-box direct sum (theta = 0: to rounding;
theta = 0.5: within the tree's accuracy), the gradients the single-box
adjoint."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1211_4406_gb300 import domain as dd  # noqa: E402


def test_factor_domains():
    assert dd.factor_domains(1) == (1, 1, 1)
    assert dd.factor_domains(2) == (2, 1, 1)
    assert dd.factor_domains(8) == (2, 2, 2)
    assert dd.factor_domains(12) == (3, 2, 2)
    assert dd.factor_domains(7) == (7, 1, 1)
    for n in range(1, 65):
        a, b, c = dd.factor_domains(n)
        assert a * b * c == n and a >= b >= c


def test_multisection_balances_samples():
    from paper_1211_4406_gb300 import inputs
    pos, _ = inputs.clustered_box(40000, 40, 9)
    g = dd.multisection(pos, 3, 2, 2)
    assert g.shape == (3, 2, 2)
    from oracle import domain as od
    own = od.owner(pos, g.xc, g.yc, g.zc)
    counts = np.bincount(own, minlength=12)
    assert counts.max() - counts.min() <= 12, counts           # equal up to rounding of the cuts
    for c in (g.xc, *g.yc, *g.zc.reshape(-1, 3)):
        assert c[0] == 0.0 and c[-1] == 1.0 and np.all(np.diff(c) >= 0)
    # clustered particles make the dense domains small
    vol = np.array([g.volume(d) for d in range(12)])
    assert vol.max() / vol.min() > 2
    assert abs(vol.sum() - 1.0) < 1e-12


def test_moving_average_is_linear_weighted_over_five_steps():
    rng = np.random.default_rng(2)
    hist = [dd.multisection(rng.random((5000, 3)), 2, 2, 1) for _ in range(7)]
    avg = dd.moving_average(hist)
    w = np.arange(1, 6) / 15.0
    want = sum(wi * h.xc for wi, h in zip(w, hist[-5:]))
    assert np.allclose(avg.xc, want, rtol=0, atol=1e-15)
    assert avg.xc[0] == 0.0 and avg.xc[-1] == 1.0
    one = dd.moving_average(hist[:1])
    assert np.array_equal(one.yc, hist[0].yc)


def test_sample_counts_follow_cost():
    assert dd.sample_counts([1.0, 1.0, 2.0], 400) == [100, 100, 200]
    assert dd.sample_counts([0.0, 0.0], 10) == [5, 5]
    assert dd.sample_counts([1e-9, 1.0], 100)[0] == 1


def test_partition_boxes_balances_and_covers():
    rng = np.random.default_rng(4)
    costs = np.exp(rng.uniform(np.log(4096), np.log(884736), 64))
    for world in (1, 2, 3, 8):
        parts = dd.partition_boxes(costs, world)
        assert sorted(b for p in parts for b in p) == list(range(64))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) - min(loads) <= costs.max()          # the LPT bound
    assert dd.partition_boxes([3.0, 1.0, 2.0], 2) == [[0], [1, 2]]
    assert dd.partition_boxes([1.0, 1.0], 4) == [[0], [1], [], []]


def _partition_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1211_4406_gb300 import domain as dom
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = np.exp(np.random.default_rng(9).uniform(8, 13, 64))   # the same on every rank
        mine = dom.partition_boxes(costs, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        out.put((rank, got, float(costs[mine].sum())))
    finally:
        dist.destroy_process_group()


def test_partition_boxes_over_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    views = [g[1] for g in got]
    assert views[0] == views[1]                                  # every rank sees the same split
    assert sorted(b for part in views[0] for b in part) == list(range(64))
    assert set(views[0][0]).isdisjoint(views[0][1])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from oracle import domain as od
    from paper_1211_4406_gb300 import domain as dom
    from paper_1211_4406_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _rank_body(rank, world, out, torch, dist, oracle, od, dom, inputs)
    except Exception:
        import traceback
        out.put((rank, "error", traceback.format_exc()))
        raise
    finally:
        dist.destroy_process_group()


def _rank_body(rank, world, out, torch, dist, oracle, od, dom, inputs):
    n, rc, eps, G = 3000, 0.08, 1e-3, 1.0
    pos_all, _ = inputs.clustered_box(n, 10, 21)
    mass_all = np.full(n, 1.0 / n)
    w_all = inputs.cotangent(n, 28).astype(np.float64)
    mine = np.arange(rank, n, world)                     # an arbitrary start: every world-th particle
    pos = torch.tensor(pos_all[mine])
    mass = torch.tensor(mass_all[mine])
    ids = torch.tensor(mine, dtype=torch.int64)
    shape = dom.factor_domains(world)

    # sampling (rank r's share in proportion to its cost) and the cuts
    counts = dom.sample_counts([1.0 + r for r in range(world)], 2000)
    rng = np.random.default_rng(100 + rank)
    pick = rng.choice(pos.shape[0], min(counts[rank], pos.shape[0]), replace=False)
    samples = dom.gather_samples(pos[pick])
    geo = dom.moving_average([dom.multisection(samples, *shape)])
    xs = [torch.empty(shape[0] + 1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(xs, torch.tensor(geo.xc))
    same_cuts = all(torch.equal(xs[0], x) for x in xs)

    # particle exchange: to the owner of each particle
    idx, cnt = od.select(pos.numpy(), geo.xc, geo.yc, geo.zc, "owner")
    p, _ = dom.alltoallv(pos[idx], cnt)
    m, _ = dom.alltoallv(mass[idx], cnt)
    i, _ = dom.alltoallv(ids[idx], cnt)
    own_ok = bool(np.all(od.owner(p.numpy(), geo.xc, geo.yc, geo.zc) == rank))

    # ghost exchange
    gidx, gcnt = od.select(p.numpy(), geo.xc, geo.yc, geo.zc, "ghosts", rank, rc)
    gp, rcnt = dom.alltoallv(p[gidx], gcnt)
    gm, _ = dom.alltoallv(m[gidx], gcnt)
    gi, _ = dom.alltoallv(i[gidx], gcnt)
    lo, hi = od.boxes(geo.xc, geo.yc, geo.zc)
    own_all = od.owner(pos_all, geo.xc, geo.yc, geo.zc)
    want_ghosts = set(np.nonzero(od.near(pos_all, lo[rank], hi[rank], rc) & (own_all != rank))[0].tolist())
    ghosts_ok = set(gi.tolist()) == want_ghosts and len(gi) == len(want_ghosts)

    # per-domain forces and adjoint over own particles followed by ghosts
    nl = p.shape[0]
    allp = np.concatenate([p.numpy(), gp.numpy()])
    allm = np.concatenate([m.numpy(), gm.numpy()])
    res = {}
    for theta in (0.0, 0.5):
        t = oracle.OracleTree(allp, allm, 8, 32)
        t.lists(rc, theta)
        res[theta] = t.list_forces(G, eps, rc)[:nl]
        if theta == 0.0:
            cot = np.zeros_like(allp)
            cot[:nl] = w_all[i.numpy()]
            grad = t.list_vjp(G, eps, rc, cot)
            back, _ = dom.alltoallv(torch.tensor(grad[nl:]), rcnt)
            gl = grad[:nl].copy()
            np.add.at(gl, gidx, back.numpy())
    out.put((rank, same_cuts, own_ok, ghosts_ok, i.numpy(), res[0.0], res[0.5], gl, len(gi)))


@pytest.mark.parametrize("world", [2, 4])
def test_one_step_over_gloo_ranks_matches_the_single_box(world):
    import oracle
    from paper_1211_4406_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for g in got:
        assert g[1] != "error", g[2]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n, rc, eps, G = 3000, 0.08, 1e-3, 1.0
    pos_all, _ = inputs.clustered_box(n, 10, 21)
    mass_all = np.full(n, 1.0 / n)
    w_all = inputs.cotangent(n, 28).astype(np.float64)
    ref = oracle.brute_force(pos_all, mass_all, G, eps, rc)
    gref = oracle.brute_vjp(pos_all, mass_all, G, eps, rc, w_all)
    acc0 = np.zeros((n, 3)); acc5 = np.zeros((n, 3)); grad = np.zeros((n, 3))
    seen = np.zeros(n, dtype=np.int64)
    for rank, same_cuts, own_ok, ghosts_ok, ids, a0, a5, g, ng in got:
        assert same_cuts and own_ok and ghosts_ok, (rank, same_cuts, own_ok, ghosts_ok)
        assert ng > 0
        seen[ids] += 1
        acc0[ids], acc5[ids], grad[ids] = a0, a5, g
    assert np.all(seen == 1)                                  # every particle owned exactly once
    nr = np.linalg.norm(ref, axis=1)
    e0 = np.linalg.norm(acc0 - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    assert e0.max() <= 1e-12, e0.max()
    e5 = np.linalg.norm(acc5 - ref, axis=1) / np.maximum(nr, 1e-6 * np.median(nr))
    assert np.sqrt(np.mean(e5 ** 2)) <= 5e-3
    scale = np.sqrt(np.mean(gref ** 2))
    assert np.abs(grad - gref).max() <= 1e-10 * scale
