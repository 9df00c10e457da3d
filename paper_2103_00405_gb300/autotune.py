"""Autotuner for the trajectory-to-hardware mapping.

Batched mode: the class thresholds (thread / warp / block per trajectory) and the
block size of the persistent kernel decide how thousands of uneven networks share
the GPU.  Single networks: the mapping (thread, warp, block, bundle) and its block
size.  Each candidate runs a short probe (a capped number of events per
trajectory, same networks and seeds) timed with CUDA events; the fastest in
events per second wins.  Choices are cached in a JSON file keyed by GPU name and
problem shape (``RANDTIME_AUTOTUNE_CACHE`` overrides the path).

Results never depend on the choice: every mapping produces bit-identical
trajectories, so tuning only changes speed.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from typing import Iterable, Optional

import numpy as np
import torch

from . import _lib as L
from . import api

BATCH_CANDIDATES = [
    dict(thread_max_m=8, warp_max_m=256, block_threads=512),
    dict(thread_max_m=4, warp_max_m=256, block_threads=512),
    dict(thread_max_m=8, warp_max_m=128, block_threads=512),
    dict(thread_max_m=8, warp_max_m=256, block_threads=256),
    dict(thread_max_m=8, warp_max_m=128, block_threads=256),
    dict(thread_max_m=8, warp_max_m=64, block_threads=256),
    dict(thread_max_m=4, warp_max_m=256, block_threads=256),
    dict(thread_max_m=8, warp_max_m=256, block_threads=128),
    dict(thread_max_m=0, warp_max_m=256, block_threads=256),
]


def cache_path() -> str:
    return os.environ.get("RANDTIME_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "randtime", "autotune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict):
    path = cache_path()
    data = _load_cache()
    data[key] = value
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def batch_key(specs, n_traj: int) -> str:
    ms = sorted(int(s.n_reactions) for s in specs)
    h = hashlib.sha1(np.asarray(ms, np.int64).tobytes()).hexdigest()[:16]
    return "batch|%s|n=%d|traj=%d|M=%s" % (_gpu(), len(ms), n_traj, h)


def _time(fn, reps: int = 2) -> float:
    fn()  # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_batch(specs, x0: torch.Tensor, t_end: torch.Tensor, n_traj: int = 1, probe_events: int = 2000,
               candidates: Optional[Iterable[dict]] = None, use_cache: bool = True, seed: int = 1) -> dict:
    """Pick the batch policy with the highest events/s on a probe capped at probe_events per trajectory."""
    key = batch_key(specs, n_traj)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit["policy"]
    results = []
    for cand in candidates or BATCH_CANDIDATES:
        try:
            b = api.Batch(specs, **cand)
        except L.RandtimeError:
            continue
        out = b.outputs(n_traj)
        ms = _time(lambda: b.run(x0, t_end, n_traj, seed=seed, max_events=probe_events, outputs=out))
        events = int(out["n_events"].sum().item())
        results.append((events / (ms / 1e3), cand, ms))
        b.close()
    results.sort(key=lambda r: -r[0])
    best = dict(results[0][1])
    _store(key, {"policy": best, "events_per_s": results[0][0], "when": time.time(),
                 "tried": [[r[1], r[0]] for r in results]})
    return best


def single_key(spec, n_traj: int) -> str:
    return "single|%s|M=%d|N=%d|traj=%d" % (_gpu(), spec.n_reactions, spec.n_species, n_traj)


def tune_single(spec, x0, t_end: float, n_traj: int, probe_events: int = 2000, use_cache: bool = True,
                seed: int = 1) -> dict:
    """Pick mapping and block size for one network."""
    key = single_key(spec, n_traj)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit["launch"]
    M = spec.n_reactions
    cands = []
    if M <= 16:
        cands += [dict(mapping=L.RT_MAP_THREAD, block_threads=b) for b in (64, 128)]
    if M <= 256:
        cands.append(dict(mapping=L.RT_MAP_WARP, block_threads=0))
    if M <= 4096:
        cands += [dict(mapping=L.RT_MAP_BLOCK, block_threads=b) for b in (128, 256, 512) if 8 * b >= M]
    cands.append(dict(mapping=L.RT_MAP_BUNDLE, block_threads=0))
    net = api.Network(spec)
    results = []
    for c in cands:
        try:
            out = {}

            def go():
                out.update(api.simulate(net, x0, t_end, n_traj, seed=seed, max_events=probe_events, outputs=out,
                                        **c))
            ms = _time(go)
        except L.RandtimeError:
            continue
        events = int(out["n_events"].sum().item())
        results.append((events / (ms / 1e3), c))
    results.sort(key=lambda r: -r[0])
    best = dict(results[0][1])
    _store(key, {"launch": best, "events_per_s": results[0][0], "when": time.time(),
                 "tried": [[r[1], r[0]] for r in results]})
    return best
