"""Benchmark: reaction events per second on GB300, all five workloads, with rooflines.

Headline (the line's `value`): the ensemble workload -- the Lotka-Volterra predator-prey
model of Table 4 (c = 10, 0.01, 10; X0 = Y0 = 1000), birth-death (0 -> A at 100,
A -> 0 at 1, A0 = 0) and dimerisation (2A -> B at 0.001, B -> 2A at 0.1, A0 = 1000),
each 2^20 trajectories to t_end = 10, one thread per trajectory, Philox seed 1,
ensemble moments of X on a 0.01 grid plus final states.  Step i simulates the
trajectory ids [i * 2^20, (i+1) * 2^20) of each network on rank 0 (other ranks take
their own disjoint blocks), and the int64 moment sums are all-reduced over ranks.

`workloads` (same JSON line, each with its own small fixed step count):
  large   -- random network N = 1e4, M = 1e6, 16 trajectories, a bundle of blocks per
             trajectory streaming P, T, a through HBM (HBM roofline, 32 B per
             channel-event); --events events per trajectory per step
  large_tree -- the same network as configured (16 trajectories x 1e6 events) in the
             absolute-time form: a thread-block cluster per trajectory, min-tree argmin
  batched -- 4096 random networks, M in [4, 4096], one graph-captured persistent launch
             (FP64-issue roofline), against one launch per network on a 512-network subset
  grad    -- M = 64, N = 16, 65536 trajectories to t_end = 5, forward with the
             log-likelihood + backward kernel (FP64-issue roofline), against the plain forward
  table3  -- the paper's own Table 3 formulation against Table 2's internal-time form on the
             Lotka-Volterra model of Fig. 1, 2^18 trajectories to t_end = 10, and on the
             gradient network (M = 64) with a warp per trajectory

Printed JSON: value = events/s of the whole job (sum over ranks of fired events / max
over ranks of the timed device time); e2e = the same metric through api.simulate with
inputs copied from pinned host memory and outputs copied back inside the timed region;
roofline for the dominant kernel of each workload; cpu_baseline = the CPU oracle on
the host cores over a bounded sample of the ensemble workload (and of the other configurations).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload all|ensemble|large|large_tree|batched|grad|table3]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_00405_gb300 import workloads as W  # noqa: E402

METRIC = "reaction events/s on 1 GB300 (plain, batched, +grad) and % of roofline"
UNIT = "events/s"
SAMPLE_DT = 0.01
# Nominal FP64 rate: 1.25 TFLOP/s counts an FMA as 2 flops, so single adds, multiplies,
# divides and conversions retire at most 0.625e12 per second.  The roofline peak used
# is the rate measured by rt_fp64_probe on the same GPU at the start of the run; the
# nominal figure is printed beside it.
FP64_OP_NOMINAL = 0.625e12
# DRAM bytes per unit of work of three roofline kernels, each from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch over the units it
# processed).  A kernel changed since its capture must have its entry set to None.
NCU_TRAFFIC = {
    "k_bundle": dict(bytes_per_unit=(77562891264 + 25620826880) / (200 * 16 * 1e6), unit="channel-event",
                     source="ncu capture of k_bundle<false>, N=1e4, M=1e6, 16 trajectories x 200 events"),
    "k_ens_small": dict(bytes_per_unit=(818944 + 0) / 16384, unit="trajectory",
                        source="ncu capture of k_ens_small<3,2,false>, 16384 Lotka-Volterra trajectories to t=10"),
    "k_lazy": dict(bytes_per_unit=(2468666880 + 874632704) / (16 * 2000), unit="event",
                   source="ncu capture of k_lazy<false>, N=1e4, M=1e6, 16 trajectories x 2000 events"),
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="all",
                    choices=["all", "ensemble", "large", "large_tree", "batched", "grad", "table3"],
                    help="all (default): the ensemble headline plus the other workloads' sub-records; "
                         "one name: that workload alone as the line's headline (profiling captures)")
    ap.add_argument("--traj", type=int, default=1 << 20, help="ensemble: trajectories per network per step")
    ap.add_argument("--cpu-sample", type=int, default=1024, help="oracle trajectories per network")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--t-end", type=float, default=10.0, help="ensemble horizon (reduced only for profiling captures)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="ensemble: steps of the end-to-end leg (0: none)")
    ap.add_argument("--skip-e2e", action="store_true", help="no end-to-end leg (the same as --e2e-steps 0)")
    ap.add_argument("--sub-steps", type=int, default=2, help="timed steps of each workload of the `workloads` object")
    ap.add_argument("--sub-warmup", type=int, default=1, help="warm-up steps of each workload of `workloads`")
    ap.add_argument("--batch-events", type=int, default=20_000, help="batched workload: event cap per network")
    ap.add_argument("--nets", type=int, default=4096, help="batched workload: networks (reduced only for captures)")
    ap.add_argument("--events", type=int, default=100_000, help="large workload: events per trajectory per step")
    ap.add_argument("--tree-events", type=int, default=1_000_000,
                    help="large_tree workload: events per trajectory per step (the configuration's 1e6)")
    ap.add_argument("--grad-traj", type=int, default=65536, help="grad workload: trajectories")
    args = ap.parse_args(argv)
    if args.skip_e2e:
        args.e2e_steps = 0
    return args


# ----------------------------------------------------------------------------------------
# Sharding and reductions over ranks (host logic; tested with gloo ranks on CPU)
# ----------------------------------------------------------------------------------------

def traj_base(rank: int, step: int, n: int) -> int:
    """First global trajectory id of a rank's step: each (rank, step) pair owns its own block of
    n ids (steps < 1000), so ranks and steps never repeat a trajectory (weak scaling)."""
    return (rank * 1000 + step) * n


def shard_range(n: int, rank: int, world: int):
    """Contiguous share [start, start + count) of n items for a rank (sizes differ by at most 1)."""
    start = n * rank // world
    return start, n * (rank + 1) // world - start


def lpt_partition(costs, world: int):
    """Longest-processing-time-first: items in decreasing cost (ties by index) go to the rank with
    the least total cost so far (ties to the lower rank).  Returns one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def batched_cost(item, cap: int) -> float:
    """Estimated work of one batched network for the partition: channels scanned per event (M)
    times the expected events, t_end times the initial total propensity sum_k c_k h_k(X0)
    (Eq. 1-2, with h as a product of binomials of the reactant counts), capped at `cap`."""
    net, x = item.net, np.asarray(item.x0, np.float64)
    h = np.ones(net.n_reactions)
    xs = x[net.reac_sp]
    coef = net.reac_coef
    np.multiply.at(h, net.reac_rxn, np.where(coef == 2, xs * (xs - 1) / 2, xs))
    events = min(float(cap), float(item.t_end) * float(np.dot(net.c, h)))
    return float(net.n_reactions) * max(events, 1.0)


def combine_over_ranks(ms: float, events: int, world: int, device=None):
    """Whole-job time (the slowest rank) and events (summed over ranks) of a timed region."""
    if world <= 1:
        return ms, events
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([int(events)], dtype=torch.int64, device=device)
    dist.all_reduce(e)
    return t.item(), int(e.item())


def allreduce_moments(tensors, world: int):
    """Exact sum over ranks of int64 moment tables (grid_sum, grid_sumsq, grid_count): integer
    addition is associative, so the result equals one process's sums over all trajectories."""
    if world <= 1:
        return
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t)


def sum_in_rank_order(t, world: int):
    """Sum of a float64 tensor over ranks, added in rank order 0, 1, ... on every rank (the same
    bits on every rank and in every run, unlike a reduction whose order the library picks)."""
    if world <= 1:
        return t.clone()
    import torch
    import torch.distributed as dist
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous())
    acc = parts[0].clone()
    for p in parts[1:]:
        acc = acc + p
    return acc


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# Roofline arithmetic
# ----------------------------------------------------------------------------------------

def dependents_per_channel(net) -> np.ndarray:
    """For every channel k, how many propensities its firing recomputes: the channels reading a
    species k changes, counted once per (changed species, reading channel) pair."""
    readers = np.zeros(net.n_species, np.int64)
    np.add.at(readers, net.reac_sp, 1)
    deps = np.zeros(net.n_reactions, np.int64)
    np.add.at(deps, net.stoi_rxn, readers[net.stoi_sp])
    return deps


def fp64_ops_per_event(net, counts):
    """Algorithmic binary64 operations of the events (Table 2 with Eq. 17, 25): per event and
    channel P-T, /a, a*dt, T+ (4); per event t+dt and P_mu+E (2); a conversion and a multiply
    for every propensity the fired channel recomputes.  counts: [M] firings over the launch.
    Returns (operations, events)."""
    deps = dependents_per_channel(net)
    M = net.n_reactions
    n = float(np.sum(counts))
    return float(n * (4 * M + 2) + 2 * float(np.dot(counts, deps))), n


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def alu_roofline(ops: float, launch_ms: float, fp64_peak: float, kernel: str, note: str):
    achieved = ops / (launch_ms / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "frac_nominal": achieved / FP64_OP_NOMINAL, "traffic": None,
            "kernel": kernel, "launch_ms": launch_ms, "ops_note": note,
            "peak_note": "binary64 add/multiply issue rate measured by rt_fp64_probe in this run (of measured); "
                         "frac_nominal: against 0.625e12 single ops/s (1.25 TFLOP/s nominal with FMA = 2)"}


# ----------------------------------------------------------------------------------------
# Reference arm: the CPU oracle
# ----------------------------------------------------------------------------------------

def cpu_baseline(cfgs, sample):
    import oracle
    threads = os.cpu_count() or 1
    ev, t0 = 0, time.perf_counter()
    for c in cfgs:
        o = oracle.run(c["net"], c["x0"], c["t_end"], sample, seed=c["seed"], max_events=c["max_events"],
                       n_threads=threads)
        ev += int(o["n_events"].sum())
    dt = time.perf_counter() - t0
    return {"value": ev / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d trajectories of each of the 3 networks to t_end=%g (%d events, %.1f s)"
                      % (sample, cfgs[0]["t_end"], ev, dt)}


def cpu_other_configs():
    """The oracle on bounded samples of the other configurations: the ensemble on one core, the
    large network (one trajectory, 200 events: each event recomputes and scans all 10^6 channels),
    the gradient network with the likelihood (8192 trajectories on every core)."""
    import oracle
    threads = os.cpu_count() or 1
    out = {}

    def timed(name, desc, fn):
        t0 = time.perf_counter()
        ev = fn()
        dt = time.perf_counter() - t0
        out[name] = {"value": ev / dt, "unit": UNIT, "cores": desc[0], "sample": "%s (%d events, %.1f s)"
                     % (desc[1], ev, dt)}

    cfgs = W.ensemble_configs(32)
    timed("ensemble_single_core", (1, "32 trajectories of each ensemble network to t_end=10, one thread"),
          lambda: sum(int(oracle.run(c["net"], c["x0"], c["t_end"], 32, seed=c["seed"], max_events=c["max_events"],
                                     n_threads=1)["n_events"].sum()) for c in cfgs))
    big = W.large_network_config(max_events=200)
    timed("large_network", (1, "1 trajectory x 200 events of the N=1e4, M=1e6 network, one thread"),
          lambda: int(oracle.run(big["net"], big["x0"], big["t_end"], 1, seed=1, max_events=200)["n_events"].sum()))
    gc = W.grad_config(8192)
    timed("gradient", (threads, "8192 trajectories of the M=64 gradient network to t_end=5 with the likelihood"),
          lambda: int(oracle.run(gc["net"], gc["x0"], gc["t_end"], 8192, seed=1, want_grad=True,
                                 n_threads=threads)["n_events"].sum()))
    return out


ENSEMBLE_WORKLOAD = ("ensemble: Lotka-Volterra (Table 4, X0=Y0=1000) + birth-death (k=100, gamma=1) "
                     "+ dimerisation (0.001/0.1, A0=1000), 2^20 trajectories each, t_end=10, "
                     "one thread per trajectory")


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, on the ensemble workload's metric and
    config, each step a bounded sample of it (--cpu-sample trajectories of each network)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfgs = W.ensemble_configs(args.traj)
    sample = args.cpu_sample
    for _ in range(args.warmup):  # untimed: loads the oracle and pages its code in
        cpu_baseline(cfgs, 8)
    vals, secs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        b = cpu_baseline(cfgs, sample)
        secs.append(time.perf_counter() - t0)
        vals.append(b["value"])
    b["value"] = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ENSEMBLE_WORKLOAD, "trajectories_per_network": args.traj, "t_end": args.t_end,
                       "sample_dt": SAMPLE_DT, "seed": 1, "max_events_per_trajectory": cfgs[0]["max_events"],
                       "parallelism": "host cores"},
            "cpu_baseline": b, "e2e": {"value": b["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------------------
# Timing helpers
# ----------------------------------------------------------------------------------------

class Ctx:
    """Per-process run context: rank, world, device, stream, measured peaks."""

    def __init__(self):
        import torch
        self.rank, self.world, self.local = dist_env()
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.current_stream()
        self.fp64_peak = None

    def barrier(self):
        import torch
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()


def timed_steps(ctx, step_fn, steps, warmup, before=None, after=None):
    """Run warmup + steps calls of step_fn(i, record) bracketed by a barrier and a synchronize;
    each timed step is measured with CUDA events on the launching stream (record(name) marks
    named points inside the step).  before(i) / after(i) run outside the timed span of timed
    step i (after(i) once its end event has completed).  Returns (per-step ms, marks, clocks)."""
    import torch
    for i in range(warmup):
        if before:
            before(100 + i)
        step_fn(100 + i, lambda name: None)
    ctx.barrier()
    sampler = ClockSampler(ctx.local).start()
    ms, marks = [], []
    for i in range(steps):
        if before:
            before(i)
        ev = {}

        def record(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(ctx.stream)
            ev[name] = e
        record("_start")
        step_fn(i, record)
        record("_end")
        ev["_end"].synchronize()
        ms.append(ev["_start"].elapsed_time(ev["_end"]))
        if after:
            after(i)
        marks.append({k: ev["_start"].elapsed_time(v) for k, v in ev.items() if not k.startswith("_")})
    ctx.barrier()
    return ms, marks, sampler.stop()


# ----------------------------------------------------------------------------------------
# Ensemble (headline)
# ----------------------------------------------------------------------------------------

def run_ensemble(args, ctx):
    import torch

    from paper_2103_00405_gb300 import _lib as L
    from paper_2103_00405_gb300 import api

    n = args.traj
    cfgs = W.ensemble_configs(n)
    for c in cfgs:
        c["t_end"] = args.t_end
    nets = [api.Network(c["net"]) for c in cfgs]
    G = api.grid_len(args.t_end, SAMPLE_DT)
    outs = []
    for c in cfgs:
        N = c["net"].n_species
        outs.append(dict(x_final=torch.empty((n, N), dtype=torch.int32, device=ctx.dev),
                         n_events=torch.empty(n, dtype=torch.int64, device=ctx.dev),
                         status=torch.empty(n, dtype=torch.int32, device=ctx.dev),
                         t_last=torch.empty(n, dtype=torch.float64, device=ctx.dev),
                         grid_sum=torch.zeros((G, N), dtype=torch.int64, device=ctx.dev),
                         grid_sumsq=torch.zeros((G, N), dtype=torch.int64, device=ctx.dev),
                         grid_count=torch.zeros(G, dtype=torch.int64, device=ctx.dev)))
    x0s = [torch.as_tensor(c["x0"], dtype=torch.int32).to(ctx.dev) for c in cfgs]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=ctx.dev)  # > L2 (129 MB)
    moments = [o[k] for o in outs for k in ("grid_sum", "grid_sumsq", "grid_count")]

    def before(i):
        flush.fill_(i & 0xFF)  # evict L2 between timed steps (outside the timed span)
        for t in moments:
            t.zero_()

    def step(i, record):
        base = traj_base(ctx.rank, i, n)
        for k, c in enumerate(cfgs):
            api.simulate(nets[k], x0s[k], c["t_end"], n, seed=c["seed"], traj_offset=base, sample_dt=SAMPLE_DT,
                         max_events=c["max_events"], grid="moments", mapping=L.RT_MAP_THREAD, outputs=outs[k])
            record("launch%d" % k)
        allreduce_moments(moments, ctx.world)  # the ensemble's one exchange: exact int64 sums

    step_events = []
    ms, marks, clocks = timed_steps(ctx, step, args.steps, args.warmup, before,
                                    after=lambda i: step_events.append(
                                        sum(int(o["n_events"].sum().item()) for o in outs)))
    dev_ms, total_events = combine_over_ranks(sum(ms), sum(step_events), ctx.world, ctx.dev)
    value = total_events / (dev_ms / 1e3)

    # dominant kernel: the Lotka-Volterra launch (launch0 of each step); its algorithmic FP64
    # operations from the firing mix of the last step's first n/16 trajectories (same ids)
    lv_ms = [m["launch0"] for m in marks]
    chk = api.simulate(api.Network(cfgs[0]["net"]), x0s[0], args.t_end, max(1, n // 16), seed=1,
                       traj_offset=traj_base(ctx.rank, args.steps - 1, n), grad=True, mapping=L.RT_MAP_THREAD,
                       max_events=cfgs[0]["max_events"])
    counts = chk["counts"].sum(0, dtype=torch.int64).cpu().numpy()
    ops_s, ev_s = fp64_ops_per_event(cfgs[0]["net"], counts)
    lv_events = int(outs[0]["n_events"].sum().item())
    roof = alu_roofline(ops_s / ev_s * lv_events, lv_ms[-1], ctx.fp64_peak, "k_ens_small<3,2,false> "
                        "(Lotka-Volterra launch)", "%.3f algorithmic FP64 ops per event (4M+2 + 2 per recomputed "
                        "propensity)" % (ops_s / ev_s))
    tr = NCU_TRAFFIC["k_ens_small"]
    roof["traffic"] = tr["bytes_per_unit"] * n if tr["bytes_per_unit"] else None
    roof["traffic_note"] = tr["source"] + ", scaled to this launch's trajectories"

    # end to end through the public API: pinned host inputs in, results back to pinned host memory
    x0_host = [torch.as_tensor(c["x0"], dtype=torch.int32).pin_memory() for c in cfgs]
    host_out = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                 for k, v in o.items() if k in ("x_final", "n_events", "status", "grid_sum", "grid_sumsq",
                                                "grid_count")} for o in outs]
    h2d = sum(x.numel() * x.element_size() for x in x0_host)
    d2h = sum(v.numel() * v.element_size() for ho in host_out for v in ho.values())
    e2e_ms, e2e_events = 0.0, 0
    for i in range(min(args.e2e_steps, args.steps)):
        flush.fill_(i & 0xFF)
        for t in moments:
            t.zero_()
        ctx.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        for k, c in enumerate(cfgs):
            xd = x0_host[k].to(ctx.dev, non_blocking=True)
            api.simulate(nets[k], xd, c["t_end"], n, seed=c["seed"], traj_offset=traj_base(ctx.rank, 50 + i, n),
                         sample_dt=SAMPLE_DT, max_events=c["max_events"], grid="moments", mapping=L.RT_MAP_THREAD,
                         outputs=outs[k])
        allreduce_moments(moments, ctx.world)
        for k in range(len(cfgs)):
            for key, hv in host_out[k].items():
                hv.copy_(outs[k][key], non_blocking=True)
        b.record(ctx.stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
        e2e_events += sum(int(ho["n_events"].sum()) for ho in host_out)
    if e2e_ms > 0:
        e2e_ms, e2e_events = combine_over_ranks(e2e_ms, e2e_events, ctx.world, ctx.dev)
    e2e_value = e2e_events / (e2e_ms / 1e3) if e2e_ms > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ctx.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ENSEMBLE_WORKLOAD, "trajectories_per_network": n, "t_end": args.t_end,
                   "sample_dt": SAMPLE_DT, "seed": 1, "max_events_per_trajectory": cfgs[0]["max_events"],
                   "parallelism": ("trajectories sharded over %d ranks, int64 moment sums all-reduced"
                                   % ctx.world) if ctx.world > 1 else "1 GPU",
                   "l2": "flushed between timed steps (512 MB write)",
                   "events_per_step": total_events / args.steps},
        "clocks": clocks,
        "gpu_launches": 3 * args.steps,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": min(args.e2e_steps, args.steps)},
    }
    if not args.no_cpu_baseline and ctx.world == 1:
        line["cpu_baseline"] = cpu_baseline(cfgs, args.cpu_sample)
        line["cpu_baseline"]["other_configs"] = cpu_other_configs()
    return line


# ----------------------------------------------------------------------------------------
# Large network (eager bundle)
# ----------------------------------------------------------------------------------------

def run_large(args, ctx, steps, warmup):
    """N = 1e4 species, M = 1e6 reactions, 16 trajectories per rank (replicas: a single
    trajectory does not shard), `--events` events each per step from a fresh start (t_end = inf),
    a bundle of blocks per trajectory streaming P, T, a through HBM."""
    import torch

    from paper_2103_00405_gb300 import _lib as L
    from paper_2103_00405_gb300 import api

    cfg = W.large_network_config(max_events=args.events)
    net, n_traj, M = cfg["net"], cfg["n_traj"], cfg["net"].n_reactions
    netg = api.Network(net)
    x0 = torch.as_tensor(cfg["x0"], dtype=torch.int32).to(ctx.dev)
    outs = {}
    step_events = []

    def step(i, record):
        o = api.simulate(netg, x0, math.inf, n_traj, seed=1, traj_offset=traj_base(ctx.rank, i, n_traj),
                         max_events=args.events, mapping=L.RT_MAP_BUNDLE, outputs=outs)
        outs.update(o)

    ms, _, clocks = timed_steps(ctx, step, steps, warmup,
                                after=lambda i: step_events.append(int(outs["n_events"].sum().item())))
    events = sum(step_events)
    dev_ms, events_all = combine_over_ranks(sum(ms), events, ctx.world, ctx.dev)
    peak, how = hbm_peak_gbs()
    per_launch_events = events / steps
    achieved = 32.0 * M * per_launch_events / (statistics.mean(ms) / 1e3) / 1e9
    tr = NCU_TRAFFIC["k_bundle"]
    return {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": dev_ms / steps,
            "config": {"workload": "large network: random mass-action N=1e4, M=1e6 uni/bimolecular, "
                                   "c~lognormal(0,1), X0~Poisson(100), 16 trajectories per rank, bundle of blocks "
                                   "per trajectory",
                       "events_per_trajectory_per_step": args.events,
                       "step": "16 fresh trajectories (new ids each step, init kernel inside the timed span) "
                               "run for %d events each; the 1e6-event runs of the configuration take 10 such "
                               "steps" % args.events,
                       "t_end": "inf", "seed": 1, "parallelism": "replicas" if ctx.world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (16 x 24 MB of P, T, a streamed per event)"},
            "events_per_step": events_all / steps, "clocks": clocks, "gpu_launches": 2 * steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (tr["bytes_per_unit"] * M * per_launch_events if tr["bytes_per_unit"] else None),
                         "traffic_note": tr["source"] + ", scaled to this launch's channel-events",
                         "kernel": "k_bundle<false>", "bytes_per_channel_event": 32, "peak_source": how}}


def distinct_dependents(net, channels) -> np.ndarray:
    """For each listed channel k, how many distinct channels (k itself included) its firing touches
    in the absolute-time form: k and every channel reading a species k changes."""
    order = np.argsort(net.reac_sp, kind="stable")
    rsp, rk = net.reac_sp[order], net.reac_rxn[order]
    start = np.searchsorted(rsp, np.arange(net.n_species + 1))
    vord = np.argsort(net.stoi_rxn, kind="stable")
    vk, vsp = net.stoi_rxn[vord], net.stoi_sp[vord]
    vstart = np.searchsorted(vk, np.arange(net.n_reactions + 1))
    out = []
    for k in np.asarray(channels).tolist():
        touched = {k}
        for sp in vsp[vstart[k]:vstart[k + 1]].tolist():
            touched.update(rk[start[sp]:start[sp + 1]].tolist())
        out.append(len(touched))
    return np.array(out, np.int64)


def run_large_tree(args, ctx, steps, warmup):
    """The large-network configuration as written -- N = 1e4, M = 1e6, 16 trajectories per rank,
    1e6 events each (t_end = inf) -- in the absolute-time form on the tree mapping: a cluster of
    CTAs per trajectory, min-tree argmin, only the channels an event touches updated."""
    import torch

    from paper_2103_00405_gb300 import _lib as L
    from paper_2103_00405_gb300 import api

    ev_per_traj = args.tree_events
    cfg = W.large_network_config(max_events=ev_per_traj)
    net, n_traj = cfg["net"], cfg["n_traj"]
    netg = api.Network(net)
    x0 = torch.as_tensor(cfg["x0"], dtype=torch.int32).to(ctx.dev)
    outs = {}
    step_events = []

    def step(i, record):
        outs.update(api.simulate(netg, x0, math.inf, n_traj, seed=1, traj_offset=traj_base(ctx.rank, i, n_traj),
                                 max_events=ev_per_traj, form=L.RT_FORM_ABSOLUTE, outputs=outs))

    ms, _, clocks = timed_steps(ctx, step, steps, warmup,
                                after=lambda i: step_events.append(int(outs["n_events"].sum().item())))
    events = sum(step_events)
    dev_ms, events_all = combine_over_ranks(sum(ms), events, ctx.world, ctx.dev)
    # algorithmic bytes per event: per touched channel its 32-byte record read and written, its
    # firing time written (8), its reader-list entry, reactant descriptor and rate read (4 + 8 + 8);
    # per event the fired channel's 32-channel group re-read (256: the fired channel was that
    # group's minimum, so the group's new minimum needs all 32 firing times)
    chk = api.simulate(netg, x0, math.inf, 1, seed=1, traj_offset=traj_base(ctx.rank, steps - 1, n_traj),
                       max_events=min(ev_per_traj, 20000), grad=True, form=L.RT_FORM_ABSOLUTE)
    counts = chk["counts"][0].cpu().numpy().astype(np.float64)
    fired = np.flatnonzero(counts)
    touched = float(np.dot(counts[fired], distinct_dependents(net, fired)) / max(1.0, counts.sum()))
    bytes_per_event = touched * (32 + 32 + 8 + 4 + 8 + 8) + 256
    peak, how = hbm_peak_gbs()
    achieved = bytes_per_event * (events / steps) / (statistics.mean(ms) / 1e3) / 1e9
    return {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": dev_ms / steps,
            "config": {"workload": "large network as configured: random mass-action N=1e4, M=1e6 uni/bimolecular, "
                                   "c~lognormal(0,1), X0~Poisson(100), 16 trajectories x %d events each per rank, "
                                   "absolute-time form (dependency graph), a thread-block cluster per trajectory, "
                                   "min-tree argmin" % ev_per_traj,
                       "t_end": "inf", "seed": 1, "parallelism": "replicas" if ctx.world > 1 else "1 GPU",
                       "l2": "per-channel state 16 x 44 MB, touched at random; no streaming"},
            "events_per_step": events_all / steps, "clocks": clocks, "gpu_launches": 2 * steps,
            "us_per_event_per_trajectory": statistics.mean(ms) * 1e3 / ev_per_traj,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (NCU_TRAFFIC["k_lazy"]["bytes_per_unit"] * events / steps
                                     if NCU_TRAFFIC["k_lazy"]["bytes_per_unit"] else None),
                         "traffic_note": NCU_TRAFFIC["k_lazy"]["source"] + ", scaled to this launch's events (random "
                                         "32-byte sectors: ~2.5x the algorithmic bytes)",
                         "kernel": "k_lazy<false>", "bytes_per_event": bytes_per_event,
                         "touched_channels_per_event": touched, "peak_source": how,
                         "note": "latency-bound: each event is a chain of dependent steps (slice minima, mailbox "
                                 "exchange, fire, touched channels, group minima); the bytes moved per event are "
                                 "under 1/700 of the internal-time scan's 32 MB, so the HBM fraction is small by "
                                 "construction; the event rate is the figure of merit"}}


def run_table3(args, ctx, steps, warmup):
    """The paper's own GPU formulation (Table 3: relative waiting times rescaled after every
    event, every propensity recomputed) against Table 2's internal-time form, on the model of the
    paper's Fig. 1 (Lotka-Volterra, Table 4 rates, X0 = Y0 = 1000), 2^18 trajectories to t_end = 10
    per step, one thread per trajectory, the same trajectories both ways; then the same on the
    gradient network (M = 64) with a warp per trajectory (Table 3's form, a lane per channel)
    against warp segments (Table 2's form)."""
    import torch

    from paper_2103_00405_gb300 import _lib as L
    from paper_2103_00405_gb300 import api

    n = 1 << 18
    cfg = W.ensemble_configs(n)[0]
    netg = api.Network(cfg["net"])
    x0 = torch.as_tensor(cfg["x0"], dtype=torch.int32).to(ctx.dev)
    res = {}
    for name, form in (("table3_rescaled", L.RT_FORM_RESCALED), ("table2_internal", L.RT_FORM_INTERNAL)):
        outs = {}
        step_events = []

        def step(i, record):
            outs.update(api.simulate(netg, x0, cfg["t_end"], n, seed=1, traj_offset=traj_base(ctx.rank, i, n),
                                     max_events=cfg["max_events"], mapping=L.RT_MAP_THREAD, form=form,
                                     outputs=outs))

        ms, _, clocks = timed_steps(ctx, step, steps, warmup,
                                    after=lambda i: step_events.append(int(outs["n_events"].sum().item())))
        dev_ms, events_all = combine_over_ranks(sum(ms), sum(step_events), ctx.world, ctx.dev)
        res[name] = {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "ms_per_step": dev_ms / steps,
                     "events_per_step": events_all / steps, "clocks": clocks,
                     "kernel": "k_ens_rescaled<3,false,true>" if form == L.RT_FORM_RESCALED
                     else "k_ens_small<3,2,false>"}
    # the same comparison on a mid-size network (the gradient workload's M = 64, N = 16): Table 3's
    # form with a lane per channel (the paper's thread-per-reaction layout) against Table 2's form
    # on warp segments, 16384 trajectories to t_end = 5
    gcfg = W.grad_config(16384)
    gnet = api.Network(gcfg["net"])
    gx0 = torch.as_tensor(gcfg["x0"], dtype=torch.int32).to(ctx.dev)
    ng = gcfg["n_traj"]
    mid = {}
    for name, form in (("table3_rescaled_warp", L.RT_FORM_RESCALED), ("table2_internal_warp", L.RT_FORM_INTERNAL)):
        outs = {}
        step_events = []

        def step(i, record):
            outs.update(api.simulate(gnet, gx0, gcfg["t_end"], ng, seed=1, traj_offset=traj_base(ctx.rank, i, ng),
                                     max_events=10**8, mapping=L.RT_MAP_WARP, form=form, outputs=outs))

        ms, _, _ = timed_steps(ctx, step, steps, warmup,
                               after=lambda i: step_events.append(int(outs["n_events"].sum().item())))
        dev_ms, events_all = combine_over_ranks(sum(ms), sum(step_events), ctx.world, ctx.dev)
        mid[name] = {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "ms_per_step": dev_ms / steps,
                     "kernel": "k_ens_rescaled_warp<2,false>" if form == L.RT_FORM_RESCALED
                     else "k_ens_warp<8,8,false>"}
    line = {"value": res["table3_rescaled"]["value"], "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": res["table3_rescaled"]["ms_per_step"],
            "config": {"workload": "Table 3's form vs Table 2's internal-time form: Lotka-Volterra (Fig. 1 model, "
                                   "Table 4 rates, X0=Y0=1000), 2^18 trajectories to t_end=10 per step, one thread "
                                   "per trajectory, the same trajectories both ways",
                       "parallelism": "trajectories sharded over ranks" if ctx.world > 1 else "1 GPU"},
            "gpu_launches": steps, "forms": res,
            "internal_over_rescaled": res["table2_internal"]["value"] / res["table3_rescaled"]["value"],
            "mid_size": {"workload": "the gradient network (M=64, N=16), 16384 trajectories to t_end=5, warp mapping",
                         "forms": mid, "internal_over_rescaled":
                         mid["table2_internal_warp"]["value"] / mid["table3_rescaled_warp"]["value"]}}
    return line


# ----------------------------------------------------------------------------------------
# Batched
# ----------------------------------------------------------------------------------------

def run_batched(args, ctx, steps, warmup):
    """4096 random networks, M ~ U{4..4096}, N = max(1, M/4), c ~ lognormal(0,1), X0 ~ Poisson(50),
    t_end ~ U[1,10], one trajectory each, capped at --batch-events events: one persistent CUDA-graph
    launch (policy from the autotuner) per rank over its longest-processing-time-first share of the
    networks, against one rt_run launch per network on a 512-network subset."""
    import torch

    from paper_2103_00405_gb300 import api, autotune

    items_all = W.batched_networks(args.nets)
    mine = lpt_partition([batched_cost(it, args.batch_events) for it in items_all], ctx.world)[ctx.rank]
    items = [items_all[i] for i in mine]
    specs = [it.net for it in items]
    sid = np.asarray(mine, np.uint32)  # each network keeps its global Philox stream
    x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).to(ctx.dev)
    t_end = torch.tensor([it.t_end for it in items], dtype=torch.float64, device=ctx.dev)
    cap = args.batch_events
    policy = autotune.tune_batch(specs, x0, t_end, 1, probe_events=max(100, cap // 20))
    batch = api.Batch(specs, stream_ids=sid, **policy)
    graph, out = batch.capture(x0, t_end, 1, seed=1, max_events=cap)
    ms, _, clocks = timed_steps(ctx, lambda i, r: graph.replay(), steps, warmup)
    ev_net = out["n_events"][:, 0].cpu().numpy()
    events = int(ev_net.sum())
    dev_ms, events_all = combine_over_ranks(sum(ms), events * steps, ctx.world, ctx.dev)

    # algorithmic FP64 operations: per event of network i, 4 M_i + 2, plus 2 per recomputed
    # propensity with the mean dependents count of the network's channels
    ops = 0.0
    for it, e in zip(items, ev_net):
        ops += float(e) * (4 * it.net.n_reactions + 2 + 2 * float(dependents_per_channel(it.net).mean()))
    roof = alu_roofline(ops, statistics.mean(ms), ctx.fp64_peak, "k_batch<false> (persistent, graph-captured)",
                        "per event of network i: 4 M_i + 2 + 2 x mean dependents of its channels")

    line = {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": dev_ms / steps,
            "config": {"workload": "batched: %d random networks, M~U{4..4096}, N=M/4, c~lognormal(0,1), "
                                   "X0~Poisson(50), t_end~U[1,10], 1 trajectory each, one persistent graph launch"
                                   % args.nets, "max_events_per_network": cap, "policy": policy,
                       "networks_this_rank": len(items),
                       "parallelism": ("networks split over %d ranks, longest processing time first"
                                       % ctx.world) if ctx.world > 1 else "1 GPU",
                       "l2": "network tables ~%d MB (about 170 B per reaction: descriptors, rates, net changes, "
                             "reader and dependent lists) read through L2; graph replays back to back"
                             % int(sum(it.net.n_reactions for it in items) * 170 / 2**20)},
            "events_per_step": events_all / steps, "clocks": clocks, "gpu_launches": steps, "roofline": roof}

    if ctx.rank == 0:
        # a 512-network subset both ways: one batch launch, and one rt_run launch per network
        # (stream_id = the network's id, so the trajectories are identical), spread over 8 streams
        sub_idx = mine[:512]
        sub = [items_all[i] for i in sub_idx]
        sbatch = api.Batch([it.net for it in sub], stream_ids=np.asarray(sub_idx, np.uint32), **policy)
        sx0 = torch.from_numpy(np.concatenate([it.x0 for it in sub])).to(ctx.dev)
        st = torch.tensor([it.t_end for it in sub], dtype=torch.float64, device=ctx.dev)
        sgraph, sout = sbatch.capture(sx0, st, 1, seed=1, max_events=cap)
        ms_sub, _, _ = timed_steps(_Solo(ctx), lambda i, r: sgraph.replay(), steps, 1)
        nets = [api.Network(it.net) for it in sub]
        x0s = [torch.as_tensor(it.x0, dtype=torch.int32).to(ctx.dev) for it in sub]
        outs = [{} for _ in sub]
        streams = [torch.cuda.Stream() for _ in range(8)]

        def per_network(i, r):
            for s_ in streams:
                s_.wait_stream(ctx.stream)
            for q, it in enumerate(sub):
                with torch.cuda.stream(streams[q % 8]):
                    api.simulate(nets[q], x0s[q], it.t_end, 1, seed=1, stream_id=int(sub_idx[q]), max_events=cap,
                                 outputs=outs[q])
            for s_ in streams:
                ctx.stream.wait_stream(s_)

        ms_plain, _, _ = timed_steps(_Solo(ctx), per_network, 1, 1)
        plain_events = sum(int(o["n_events"].sum().item()) for o in outs)
        sub_events = int(sout["n_events"].sum().item())
        assert plain_events == sub_events, (plain_events, sub_events)
        line["subset_512"] = {"batched_events_per_s": sub_events / (statistics.mean(ms_sub) / 1e3),
                              "per_network_launches_events_per_s": plain_events / (statistics.mean(ms_plain) / 1e3),
                              "unit": UNIT, "events": sub_events, "per_network_streams": 8}
    return line


class _Solo:
    """A single-rank view of a context (for comparisons that only rank 0 runs)."""

    def __init__(self, ctx):
        self.rank, self.world, self.local = 0, 1, ctx.local
        self.dev, self.stream = ctx.dev, ctx.stream

    def barrier(self):
        import torch
        torch.cuda.synchronize()


# ----------------------------------------------------------------------------------------
# Gradient
# ----------------------------------------------------------------------------------------

def run_grad(args, ctx, steps, warmup):
    """Random network M = 64, N = 16, c ~ lognormal(0, 0.5), X0 ~ Poisson(200), 65536 trajectories
    to t_end = 5 (sharded over ranks by global id): forward with the log-likelihood plus the
    backward kernel, grad_c summed over ranks in rank order; against the plain forward."""
    import torch

    from paper_2103_00405_gb300 import api

    cfg = W.grad_config(args.grad_traj)
    net = cfg["net"]
    start, n = shard_range(cfg["n_traj"], ctx.rank, ctx.world)
    netg = api.Network(net)
    x0 = torch.as_tensor(cfg["x0"], dtype=torch.int32).to(ctx.dev)
    out_plain, out_grad = {}, {}
    ones = torch.ones(n, dtype=torch.float64, device=ctx.dev)
    state = {}

    def fwd_bwd(i, record):
        o = api.simulate(netg, x0, cfg["t_end"], n, seed=1, traj_offset=start, max_events=10**8, grad=True,
                         outputs=out_grad)
        record("forward")
        g = api.loglik_backward(netg, ones, o["counts"], o["t_internal"])
        state["g"] = sum_in_rank_order(g, ctx.world)

    def fwd_plain(i, record):
        api.simulate(netg, x0, cfg["t_end"], n, seed=1, traj_offset=start, max_events=10**8, outputs=out_plain)

    ms, marks, clocks = timed_steps(ctx, fwd_bwd, steps, warmup)
    ms_plain, _, _ = timed_steps(ctx, fwd_plain, steps, warmup)
    events = int(out_grad["n_events"].sum().item())
    assert events == int(out_plain["n_events"].sum().item())
    dev_ms, events_all = combine_over_ranks(sum(ms), events * steps, ctx.world, ctx.dev)
    pms, _ = combine_over_ranks(sum(ms_plain), 0, ctx.world, ctx.dev)
    counts = out_grad["counts"].sum(0, dtype=torch.int64).cpu().numpy()
    ops, ev = fp64_ops_per_event(net, counts)
    fwd_ms = statistics.mean(m["forward"] for m in marks)
    roof = alu_roofline(ops, fwd_ms, ctx.fp64_peak, "k_ens_warp<8,8,true> (8 lanes per trajectory, forward with the log-likelihood)",
                        "%.1f algorithmic FP64 ops per event (4M+2 + 2 per recomputed propensity; the "
                        "fixed-point logarithms are integer work)" % (ops / ev))
    return {"value": events_all / (dev_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": dev_ms / steps,
            "config": {"workload": "gradient: random network M=64, N=16, c~lognormal(0,0.5), X0~Poisson(200), "
                                   "%d trajectories to t_end=5, forward with log-likelihood + backward kernel"
                                   % cfg["n_traj"],
                       "parallelism": ("trajectories sharded over %d ranks, grad_c summed in rank order"
                                       % ctx.world) if ctx.world > 1 else "1 GPU",
                       "l2": "state in registers; outputs 64 MB written per step"},
            "events_per_step": events_all / steps, "clocks": clocks, "gpu_launches": 2 * steps,
            "backward_ms": statistics.mean(m_ - m["forward"] for m_, m in zip(ms, marks)),
            "roofline": roof,
            "plain_forward": {"value": events_all / (pms / 1e3), "unit": UNIT, "ms_per_step": pms / steps}}


# ----------------------------------------------------------------------------------------

def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ctx = Ctx()
    if ctx.world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_00405_gb300 import api
    ctx.fp64_peak = api.fp64_probe()
    sub = dict(steps=args.sub_steps, warmup=args.sub_warmup)
    if args.workload in ("all", "ensemble"):
        line = run_ensemble(args, ctx)
        if args.workload == "all":
            line["workloads"] = {"large": run_large(args, ctx, **sub), "large_tree": run_large_tree(args, ctx, **sub),
                                 "batched": run_batched(args, ctx, **sub), "grad": run_grad(args, ctx, **sub),
                                 "table3": run_table3(args, ctx, **sub)}
    else:
        fn = {"large": run_large, "large_tree": run_large_tree, "batched": run_batched, "grad": run_grad,
              "table3": run_table3}[args.workload]
        rec = fn(args, ctx, args.steps, args.warmup)
        line = {"metric": METRIC, "value": rec.pop("value"), "unit": UNIT, "n_gpus": ctx.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": rec.pop("ms_per_step"), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
        line.update(rec)
    line["fp64_peak_ops_per_s"] = ctx.fp64_peak
    if ctx.rank == 0:
        print(json.dumps(line))
    if ctx.world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
