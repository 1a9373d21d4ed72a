"""Multi-rank host logic of the replica bench (world size 2, gloo, CPU).

Each rank solves its own seeded problem; the timed region is bracketed by barriers and
the job's time is the slowest rank's.  Here the ranks run a stand-in step on the CPU
(rank 1 sleeps longer), so the max-reduction, the throughput and the per-rank seeds can be
checked without a GPU.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_00735_gb300 import inputs
from paper_2511_00735_gb300 import replicas as RP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        delay = 0.05 * (1 + 2 * rank)  # rank 1 is the slow replica
        clock = RP.WallClock()
        ms, wall_ms, outs = RP.timed(lambda: (__import__("time").sleep(delay), rank)[1], 3, clock, dist=dist)
        prob = inputs.fp64_64x64(seed=RP.seed_for_rank(rank), nrhs=2)
        seeds = [None] * world
        dist.all_gather_object(seeds, (RP.seed_for_rank(rank), prob.bumps[0]))
        out.put((rank, ms, wall_ms, outs, RP.job_throughput(prob.nrhs, 3, world, ms), seeds))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, w0, o0, v0, s0), (r1, ms1, w1, o1, v1, s1) = res
    # both ranks hold the same reduced times: the slow rank's (3 x 0.15 s)
    assert ms0 == ms1 and w0 == w1
    assert 450.0 <= ms0 < 2000.0 and w0 >= ms0 - 1.0
    assert o0 == [0, 0, 0] and o1 == [1, 1, 1]
    # whole-job throughput: both ranks' units over the slowest rank's time
    assert v0 == v1 == pytest.approx(3 * 2 * 2 / (ms0 / 1e3))
    # every replica solves a different seeded problem
    assert s0 == s1 and s0[0][0] != s0[1][0] and s0[0][1] != s0[1][1]


def test_single_process_needs_no_collective():
    clock = RP.WallClock()
    ms, wall, outs = RP.timed(lambda: 7, 4, clock)
    assert outs == [7, 7, 7, 7] and 0.0 <= ms <= wall + 1.0
    assert RP.max_over_ranks(3.5) == 3.5
    assert RP.job_throughput(16, 3, 1, 1500.0) == pytest.approx(32.0)
    assert RP.seed_for_rank(0) == 1 and RP.seed_for_rank(3) == 4
