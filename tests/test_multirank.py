"""The multi-rank paths of the benchmark on CPU: two gloo ranks, each simulating its share with
the CPU oracle.

Trajectories and networks are independent (Sec. 5), so the workloads shard with no exchange on
the simulation path:
  * ensemble: each (rank, step) owns a block of global trajectory ids (`bench.traj_base`); the
    int64 moment sums are all-reduced exactly (`bench.allreduce_moments`);
  * batched: networks are split longest-processing-time-first (`bench.lpt_partition`) and keep
    their global Philox stream, so every network's trajectory equals the single-process one;
  * gradient: trajectories are split by global id (`bench.shard_range`); grad_c is summed over
    ranks in rank order (`bench.sum_in_rank_order`), the same bits on every rank and every run;
  * large network: replicas (distinct trajectory ids per rank), events summed, time the maximum.
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


def _spawn(target, world=2, args=()):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + tuple(args)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(got, key=lambda g: g[0])


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _moments(grid):
    """int64 sums over trajectories of X and X^2 per grid point, and the known-point counts."""
    g = grid.astype(np.int64)
    known = (g >= 0).all(axis=2)
    gs = np.where(known[:, :, None], g, 0)
    return gs.sum(0), (gs * gs).sum(0), known.sum(0).astype(np.int64)


ENS_N, ENS_T, ENS_DT = 20, 1.0, 0.1


def _ensemble_rank(rank, world, port, q):
    import torch
    dist = _init(rank, world, port)
    try:
        cfg = W.ensemble_configs(ENS_N)[2]  # dimerisation
        base = bench.traj_base(rank, 0, ENS_N)
        o = oracle.run(cfg["net"], cfg["x0"], ENS_T, ENS_N, seed=1, traj_offset=base, sample_dt=ENS_DT,
                       want_grid=True, n_threads=1)
        tabs = [torch.from_numpy(m.copy()) for m in _moments(o["grid"])]
        bench.allreduce_moments(tabs, world)
        q.put((rank, base, [t.numpy() for t in tabs]))
    finally:
        dist.destroy_process_group()


def test_ensemble_moment_sums_all_reduced_exactly():
    got = _spawn(_ensemble_rank)
    cfg = W.ensemble_configs(ENS_N)[2]
    ref = [np.zeros_like(m) for m in got[0][2]]
    for _, base, _ in got:  # one process over the same global ids
        o = oracle.run(cfg["net"], cfg["x0"], ENS_T, ENS_N, seed=1, traj_offset=base, sample_dt=ENS_DT,
                       want_grid=True, n_threads=1)
        for r, m in zip(ref, _moments(o["grid"])):
            r += m
    for _, _, tabs in got:
        for a, b in zip(tabs, ref):
            assert a.dtype == np.int64 and np.array_equal(a, b)


N_NETS, CAP = 12, 400


def _batched_rank(rank, world, port, q):
    dist = _init(rank, world, port)
    try:
        items = W.batched_networks(N_NETS, m_lo=2, m_hi=40, seed=77, t_lo=0.05, t_hi=0.2)
        mine = bench.lpt_partition([bench.batched_cost(it, CAP) for it in items], world)[rank]
        res = {}
        for i in mine:  # each network keeps its global index as Philox stream
            o = oracle.run(items[i].net, items[i].x0, items[i].t_end, 2, seed=1, stream_id=i, max_events=CAP,
                           n_threads=1)
            res[i] = (o["x_final"].copy(), o["n_events"].copy())
        q.put((rank, mine, res))
    finally:
        dist.destroy_process_group()


def test_batched_networks_split_longest_first_keep_their_streams():
    got = _spawn(_batched_rank)
    parts = [g[1] for g in got]
    assert sorted(parts[0] + parts[1]) == list(range(N_NETS)) and not set(parts[0]) & set(parts[1])
    items = W.batched_networks(N_NETS, m_lo=2, m_hi=40, seed=77, t_lo=0.05, t_hi=0.2)
    for _, _, res in got:
        for i, (xf, ne) in res.items():
            o = oracle.run(items[i].net, items[i].x0, items[i].t_end, 2, seed=1, stream_id=i, max_events=CAP,
                           n_threads=1)
            assert np.array_equal(o["x_final"], xf) and np.array_equal(o["n_events"], ne)


def test_lpt_partition_balances_and_is_deterministic():
    costs = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4]
    p = bench.lpt_partition(costs, 3)
    assert sorted(sum(p, [])) == list(range(len(costs)))
    loads = [sum(costs[i] for i in part) for part in p]
    assert max(loads) - min(loads) <= max(costs) and p == bench.lpt_partition(costs, 3)
    assert bench.lpt_partition(costs, 1) == [list(range(len(costs)))]


GRAD_N = 30


def _grad_rank(rank, world, port, q):
    import torch
    dist = _init(rank, world, port)
    try:
        cfg = W.grad_config(GRAD_N)
        start, n = bench.shard_range(GRAD_N, rank, world)
        o = oracle.run(cfg["net"], cfg["x0"], 0.05, n, seed=1, traj_offset=start, want_grad=True, n_threads=1)
        g = oracle.loglik_backward(np.ones(n), o["counts"], o["t_internal"], cfg["net"].c)
        tot = bench.sum_in_rank_order(torch.from_numpy(g), world)
        q.put((rank, start, n, g, tot.numpy()))
    finally:
        dist.destroy_process_group()


def test_gradient_sharded_and_summed_in_rank_order():
    got = _spawn(_grad_rank)
    assert got[0][1] == 0 and got[0][2] + got[1][2] == GRAD_N and got[1][1] == got[0][2]
    expect = got[0][3] + got[1][3]  # rank 0's partial, then rank 1's
    for _, _, _, _, tot in got:
        assert np.array_equal(tot.view(np.int64), expect.view(np.int64))
    cfg = W.grad_config(GRAD_N)
    o = oracle.run(cfg["net"], cfg["x0"], 0.05, GRAD_N, seed=1, want_grad=True, n_threads=1)
    single = oracle.loglik_backward(np.ones(GRAD_N), o["counts"], o["t_internal"], cfg["net"].c)
    scale = np.maximum(np.abs(single), o["counts"].sum(0) / cfg["net"].c)
    assert np.all(np.abs(got[0][4] - single) <= 1e-12 * np.maximum(scale, 1.0))


def test_shard_range_covers_every_item_once():
    for n in (0, 1, 7, 65536):
        for world in (1, 2, 3, 8):
            spans = [bench.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == n
            for (s0, c0), (s1, _) in zip(spans, spans[1:]):
                assert s0 + c0 == s1


if __name__ == "__main__":  # pragma: no cover
    pytest.main([__file__, "-q"])
