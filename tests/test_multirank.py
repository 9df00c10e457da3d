"""The multi-rank path of the benchmark on CPU: two gloo ranks.

Trajectories are independent, so N ranks shard them with no collective on the data path: each
(rank, step) owns its own block of global trajectory ids (`bench.traj_base`), and only the timing
(max over ranks) and the event count (sum) are reduced (`bench.combine_over_ranks`).  Here each
rank simulates its shard with the CPU oracle; the test checks that the shards are disjoint, that
the reduction gives the slowest rank's time and the summed events, and that a sharded trajectory
is the same trajectory a single process gets for that global id (the Philox counter carries the
id, so sharding changes nothing about the sample).
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import bench
import oracle
from paper_2103_00405_gb300 import workloads as W

N_PER = 24
STEPS = 2
T_END = 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = W.birth_death()
        bases, finals, events = [], [], 0
        for i in range(STEPS):
            base = bench.traj_base(rank, i, N_PER)
            o = oracle.run(net, np.array([0], np.int32), T_END, N_PER, seed=1, traj_offset=base, n_threads=1)
            bases.append(base)
            finals.append(o["x_final"][:, 0].copy())
            events += int(o["n_events"].sum())
        ms = 10.0 + 5.0 * rank  # a stand-in for this rank's measured device time
        job_ms, job_events = bench.combine_over_ranks(ms, events, world)
        q.put((rank, bases, finals, events, job_ms, job_events))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_trajectories_and_reduce_time_and_events():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    ids = [set(range(b, b + N_PER)) for _, bases, *_ in got for b in bases]
    assert sum(len(s) for s in ids) == len(set().union(*ids)), "ranks or steps repeat trajectory ids"
    total = sum(g[3] for g in got)
    for rank, bases, finals, events, job_ms, job_events in got:
        assert job_ms == 15.0 and job_events == total  # slowest rank's time, summed events, on every rank
    # a sharded trajectory equals the one a single process simulates for the same global id
    net = W.birth_death()
    rank, bases, finals = got[1][0], got[1][1], got[1][2]
    for b, xf in zip(bases, finals):
        o = oracle.run(net, np.array([0], np.int32), T_END, 1, seed=1, traj_offset=b + 5, n_threads=1)
        assert o["x_final"][0, 0] == xf[5]


def test_trajectory_blocks_are_disjoint_for_any_rank_and_step():
    seen = set()
    n = 7
    for rank in range(8):
        for step in list(range(20)) + [50, 51, 100, 101, 102]:
            ids = set(range(bench.traj_base(rank, step, n), bench.traj_base(rank, step, n) + n))
            assert not (ids & seen)
            seen |= ids


def test_single_rank_reduction_is_the_identity():
    assert bench.combine_over_ranks(12.5, 99, 1) == (12.5, 99)


if __name__ == "__main__":  # pragma: no cover
    pytest.main([__file__, "-q"])
