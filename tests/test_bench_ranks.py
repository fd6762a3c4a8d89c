"""Host-side logic of bench.py for N > 1 ranks, on CPU with the gloo backend
(world size 2): the max-over-ranks reduction of the timed totals, the
whole-job rate, and the reference arm's rank-0-only rule."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r reports timed totals (ms) that differ per rank
        tot = bench.max_over_ranks([100.0 + 10 * rank, 200.0 - 50 * rank])
        rate = bench.whole_job_rate(world, 1000, 4, tot[0])
        # ranks with unequal shares of the work (the batched boxes): the sum
        units = bench.sum_over_ranks([1000.0 + 500 * rank])
        dist.barrier()
        out.put((rank, tot, rate, units))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo_world2():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, rate, units in res:
        # every rank sees the slowest rank's totals and the sum of the shares
        assert tot == [110.0, 200.0]
        assert units == [2500.0]
        # 2 ranks x 1000 units x 4 steps over 110 ms
        assert rate == pytest.approx(2 * 1000 * 4 / 0.110)


def test_max_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.whole_job_rate(1, 10, 2, 20.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps = 1
        warmup = 0
    bench.run_reference(A(), rank=1, world=2)      # must return at once, print nothing
    assert capsys.readouterr().out == ""
