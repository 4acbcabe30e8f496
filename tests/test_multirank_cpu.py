"""The multi-GPU path's host logic on CPU: the longest-processing-time partition of independent
(system, k-point) units, and the only cross-rank communication (the slowest rank's time, the
work all ranks did), run as two gloo ranks on 127.0.0.1."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

from paper_2507_08578_gb300 import multi as MR


def test_lpt_partition_properties():
    rng = np.random.default_rng(3)
    costs = list(rng.uniform(1, 100, 57))
    for n in (1, 2, 3, 8, 64):
        parts = MR.lpt_partition(costs, n)
        assert len(parts) == n
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))  # every unit exactly once
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy LPT: the most loaded rank exceeds the least loaded by at most one unit's cost
        assert max(loads) - min(loads) <= max(costs) + 1e-9
        assert parts == MR.lpt_partition(costs, n)  # deterministic
    # the classic LPT example: 2 ranks, costs 3,3,2,2,2 -> loads 7 and 5
    parts = MR.lpt_partition([3, 3, 2, 2, 2], 2)
    assert sorted(sum([3, 3, 2, 2, 2][i] for i in p) for p in parts) == [5, 7]
    with pytest.raises(ValueError):
        MR.lpt_partition([1.0], 0)


def test_cost_model():
    # the sphere estimate is within a few percent of the exact count of config 1 (1503)
    assert abs(MR.npw_estimate(1000.0, 10.0) - 1503) / 1503 < 0.05
    assert MR.unit_cost(1000, 16, 10) == 1000 * 20 * 11 + 20 ** 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.5][rank]
        done = [10.0, 30.0][rank]
        costs = [5.0, 1.0, 4.0, 2.0, 3.0, 3.0]
        mine = MR.lpt_partition(costs, world)[rank]
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        q.put((rank, MR.max_over_ranks(seconds, dist), MR.sum_over_ranks(done, dist),
               MR.whole_job_rate(done, seconds, dist), everyone))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, total, rate, everyone in out:
        assert mx == 2.5 and total == 40.0 and rate == 16.0
        flat = sorted(i for part in everyone for i in part)
        assert flat == list(range(6))  # the ranks' shares partition the units
    assert out[0][4] == out[1][4]  # every rank computed the same partition
