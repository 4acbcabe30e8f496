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


def _units():
    """(system, k-point) units of a few small cells (the solver on CPU is the oracle)."""
    import workloads as W
    systems = [W.tiny_system(a=6.0, ecut=2.0, natom=2, seed=41, kpts=W.SHIFTED_222[:2]),
               W.tiny_system(a=6.5, ecut=2.5, natom=3, seed=42, kpts=W.SHIFTED_222[:3]),
               W.tiny_system(a=5.5, ecut=2.0, natom=1, seed=43)]
    return systems, [(j, ik) for j, s in enumerate(systems) for ik in range(len(s.kpts))]


def _solve_unit(systems, unit, nband=6):
    import oracle as O
    j, ik = unit
    return O.all_eigenvalues(O.build_problem(systems[j], ik).dense())[:nband]


def _solve_rank(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        systems, units = _units()
        costs = [MR.unit_cost(int(MR.npw_estimate(abs(np.linalg.det(systems[j].lattice)), systems[j].ecut)),
                              systems[j].nband, 10) for j, _ in units]
        mine = {u: _solve_unit(systems, units[u]) for u in MR.lpt_partition(costs, world)[rank]}
        allres = MR.gather_results(mine, dist)
        q.put((rank, sorted(mine), {u: r.tolist() for u, r in allres.items()}))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_solve_disjoint_units_and_gather():
    """Two ranks solve disjoint shares of the units (LPT partition) and gather: the union equals
    the single-process results unit for unit, and every unit was solved exactly once."""
    systems, units = _units()
    single = {u: _solve_unit(systems, units[u]) for u in range(len(units))}
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [set(o[1]) for o in out]
    assert not (shares[0] & shares[1]) and shares[0] | shares[1] == set(range(len(units)))
    for _, _, allres in out:
        assert sorted(allres) == list(range(len(units)))
        for u, r in allres.items():
            assert np.array_equal(np.array(r), single[u])
    with pytest.raises(ValueError):
        MR.gather_results({0: 1}, _TwoRanksSameUnit())


class _TwoRanksSameUnit:
    """A stand-in group whose two ranks both report unit 0 (a partition bug)."""

    def get_world_size(self):
        return 2

    def all_gather_object(self, parts, obj):
        parts[0] = dict(obj)
        parts[1] = dict(obj)
