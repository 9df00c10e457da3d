"""High-level Python API over librandtime (PyTorch for device memory and streams).

Everything that simulates runs in the library's CUDA kernels; this module only
allocates torch tensors, fills the C structs and calls the C ABI.

  Network(net)                    -- a packed network on the current CUDA device
  simulate(...)                   -- run trajectories (Table 2 of the paper), torch outputs
  LogLik.apply(c, ...)            -- path log-likelihood with a backward kernel for d/dc
  draw_exp1 / log_eval / philox   -- the library's random draws and logarithm
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from .workloads import Network as NetworkSpec


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Network:
    """A network packed and copied to the current CUDA device (rt_network_create)."""

    def __init__(self, spec: NetworkSpec, c=None):
        self.lib = L.load()
        self.spec = spec if c is None else spec.with_rates(np.asarray(c, dtype=np.float64))
        s = self.spec
        h = ctypes.c_void_p()
        arrs = [s.reac_rxn, s.reac_sp, s.reac_coef, s.stoi_rxn, s.stoi_sp, s.stoi_delta]
        p = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
        L.check(self.lib.rt_network_create(s.n_species, s.n_reactions, len(s.reac_rxn), p[0], p[1], p[2],
                                           len(s.stoi_rxn), p[3], p[4], p[5],
                                           s.c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
                "rt_network_create")
        self.handle = h
        self.N, self.M = s.n_species, s.n_reactions
        self.device = torch.cuda.current_device()

    def set_enabled(self, enabled=None):
        """Forbid channels to fire (enabled[k] == 0): their internal times stay frozen (Table 2's
        note on boundary conditions).  None enables every channel."""
        en = None if enabled is None else np.ascontiguousarray(enabled, dtype=np.uint8)
        if en is not None and en.shape != (self.M,):
            raise ValueError("enabled must have one entry per reaction")
        torch.cuda.synchronize(self.device)  # the table is rewritten in place: no launch may still read it
        L.check(self.lib.rt_network_set_enabled(self.handle, None if en is None else en.ctypes.data_as(ctypes.c_void_p)),
                "rt_network_set_enabled")
        return self

    def set_rate_slopes(self, beta=None):
        """Time-dependent rates c_k(t) = c_k (1 + beta_k t), beta_k >= 0 (Sec. 6, Eq. 29); None
        returns to constant rates."""
        b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
        if b is not None and b.shape != (self.M,):
            raise ValueError("beta must have one entry per reaction")
        torch.cuda.synchronize(self.device)  # the slopes are rewritten in place: no launch may still read them
        L.check(self.lib.rt_network_set_rate_slopes(self.handle, None if b is None else b.ctypes.data_as(ctypes.c_void_p)),
                "rt_network_set_rate_slopes")
        return self

    def info(self):
        n, m, md = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nz = ctypes.c_int64()
        L.check(self.lib.rt_network_info(self.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(md),
                                         ctypes.byref(nz)), "rt_network_info")
        return dict(n_species=n.value, n_reactions=m.value, max_dependents=md.value, n_dependency_nz=nz.value)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rt_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_cfg(mapping: Optional[int] = None, block_threads: int = 0, ctas_per_traj: int = 0,
               lanes_per_traj: int = 0):
    return L.rt_launch_cfg(L.RT_MAP_AUTO if mapping is None else int(mapping), int(block_threads),
                           int(ctas_per_traj), int(lanes_per_traj))


def grid_len(t_end: float, sample_dt: float) -> int:
    return int(L.load().rt_grid_len(float(t_end), float(sample_dt)))


def simulate(net: Network, x0, t_end: float, n_traj: int, seed: int = 1, stream_id: int = 0,
             traj_offset: int = 0, max_events: int = (1 << 31) - 1, sample_dt: float = 0.0,
             grid: str = "none", grad: bool = False, mapping: Optional[int] = None, block_threads: int = 0,
             ctas_per_traj: int = 0, trace_len: int = 0, form: int = 0, lanes_per_traj: int = 0,
             outputs: Optional[dict] = None) -> dict:
    """Simulate n_traj trajectories; returns a dict of CUDA tensors.

    x0: [N] or [n_traj, N] int32 (numpy, list or tensor; copied to the device if needed).
    grid: "none", "traj" (per-trajectory [n_traj, G, N]) or "moments" (sums over
    trajectories of X and X^2 per grid point, plus counts).
    grad: also return loglik [n_traj], counts [n_traj, M], t_internal [n_traj, M].
    trace_len: also return trace_mu [n_traj, trace_len] (fired channel of each of the first
    trace_len events, -1 after the last) and trace_t (event times, 0 after the last).
    form: L.RT_FORM_INTERNAL (Table 2 in internal times) or L.RT_FORM_ABSOLUTE (absolute firing
    times with the dependency graph; runs on the tree mapping).
    outputs: optional dict of preallocated tensors (same keys) to write into; missing entries are
    allocated and added to it.
    """
    lib = L.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    N, M = net.N, net.M
    x0t = torch.as_tensor(x0, dtype=torch.int32)
    if x0t.device != dev:
        x0t = x0t.to(dev)
    x0t = x0t.contiguous()
    per = 1 if x0t.dim() == 2 else 0
    if per and x0t.shape[0] != n_traj:
        raise ValueError("per-trajectory x0 must have n_traj rows")
    G = grid_len(t_end, sample_dt) if grid != "none" else 0
    out = outputs if outputs is not None else {}  # filled in place when the caller passes a dict

    def get(name, shape, dtype, zero=False):
        if name not in out:
            out[name] = (torch.zeros if zero else torch.empty)(shape, dtype=dtype, device=dev)
        return out[name]

    o = L.rt_outputs()
    o.x_final_dev = _ptr(get("x_final", (n_traj, N), torch.int32))
    o.n_events_dev = _ptr(get("n_events", (n_traj,), torch.int64))
    o.status_dev = _ptr(get("status", (n_traj,), torch.int32))
    o.t_last_dev = _ptr(get("t_last", (n_traj,), torch.float64))
    if grid == "traj":
        o.grid_dev = _ptr(get("grid", (n_traj, G, N), torch.int32))
    elif grid == "moments":
        o.grid_sum_dev = _ptr(get("grid_sum", (G, N), torch.int64, True))
        o.grid_sumsq_dev = _ptr(get("grid_sumsq", (G, N), torch.int64, True))
        o.grid_count_dev = _ptr(get("grid_count", (G,), torch.int64, True))
    elif grid != "none":
        raise ValueError("grid must be 'none', 'traj' or 'moments'")
    if grad:
        o.loglik_dev = _ptr(get("loglik", (n_traj,), torch.float64))
        o.counts_dev = _ptr(get("counts", (n_traj, M), torch.int32))
        o.t_internal_dev = _ptr(get("t_internal", (n_traj, M), torch.float64))

    if trace_len:
        o.trace_len = int(trace_len)
        o.trace_mu_dev = _ptr(get("trace_mu", (n_traj, int(trace_len)), torch.int32))
        o.trace_t_dev = _ptr(get("trace_t", (n_traj, int(trace_len)), torch.float64))

    p = L.rt_run_params(_ptr(x0t), per, int(stream_id), float(t_end), int(max_events), int(seed) & (2**64 - 1),
                        int(n_traj), int(traj_offset), float(sample_dt), int(form), 0)
    cfg = launch_cfg(mapping, block_threads, ctas_per_traj, lanes_per_traj)
    nbytes = ctypes.c_size_t(0)
    L.check(lib.rt_workspace_bytes(net.handle, ctypes.byref(p), ctypes.byref(cfg), ctypes.byref(nbytes)),
            "rt_workspace_bytes")
    ws = out.get("_workspace")
    if nbytes.value and (ws is None or ws.numel() < nbytes.value):
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    if not nbytes.value:
        ws = None
    L.check(lib.rt_run(net.handle, ctypes.byref(p), ctypes.byref(o), ctypes.byref(cfg), _ptr(ws), nbytes.value,
                       _stream()), "rt_run")
    out["_x0"] = x0t  # keep inputs alive until the stream has consumed them
    if ws is not None:
        out["_workspace"] = ws
    return out


def loglik_backward(net: Network, grad_ll: torch.Tensor, counts: torch.Tensor, t_internal: torch.Tensor):
    lib = L.load()
    grad_c = torch.empty(net.M, dtype=torch.float64, device=counts.device)
    L.check(lib.rt_loglik_backward(net.handle, counts.shape[0], _ptr(grad_ll.contiguous()), _ptr(counts),
                                   _ptr(t_internal), _ptr(grad_c), _stream()), "rt_loglik_backward")
    return grad_c


class LogLik(torch.autograd.Function):
    """Trajectory log-likelihoods l_j(c) = sum ln a_mu - sum_k T_k(t_end) (Eq. 16-18), with
    d l_j / d c_k = (n_jk - T_jk(t_end)) / c_k computed by the backward kernel.

    forward(c [M] float64, spec, x0, t_end, n_traj, seed, stream_id, max_events) -> l [n_traj]
    """

    @staticmethod
    def forward(ctx, c, spec, x0, t_end, n_traj, seed=1, stream_id=0, max_events=(1 << 31) - 1):
        net = Network(spec, c.detach().cpu().numpy())
        out = simulate(net, x0, t_end, n_traj, seed=seed, stream_id=stream_id, max_events=max_events, grad=True)
        ctx.net = net
        ctx.c_device = c.device
        ctx.save_for_backward(out["counts"], out["t_internal"])
        ctx.out = out
        return out["loglik"]

    @staticmethod
    def backward(ctx, grad_ll):
        counts, t_internal = ctx.saved_tensors
        g = loglik_backward(ctx.net, grad_ll.to(device=counts.device, dtype=torch.float64), counts, t_internal)
        return g.to(ctx.c_device), None, None, None, None, None, None, None


class Batch:
    """Many networks in one persistent launch (rt_batch_create / rt_batch_run).

    Network i draws its random numbers with stream_id = stream_ids[i] (default i), so its
    trajectories are those of ``simulate(Network(specs[i]), ..., stream_id=stream_ids[i])``.
    """

    def __init__(self, specs, thread_max_m: int = 8, warp_max_m: int = 256, block_threads: int = 512,
                 blocks_per_sm: int = 0, stream_ids=None, enabled=None):
        self.lib = L.load()
        nets = [Network(s) for s in specs]
        if enabled is not None:  # per network: forbidden channels (Network.set_enabled), or None
            for n, e in zip(nets, enabled):
                if e is not None:
                    n.set_enabled(e)
        arr = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
        pol = L.rt_batch_policy(thread_max_m, warp_max_m, block_threads, blocks_per_sm)
        h = ctypes.c_void_p()
        sid = None
        if stream_ids is not None:
            sid = np.ascontiguousarray(stream_ids, dtype=np.uint32)
            if sid.shape != (len(nets),):
                raise ValueError("stream_ids must have one entry per network")
        self.stream_ids = sid if sid is not None else np.arange(len(nets), dtype=np.uint32)
        L.check(self.lib.rt_batch_create(len(nets), ctypes.cast(arr, ctypes.c_void_p),
                                         None if sid is None else sid.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(pol), ctypes.byref(h)), "rt_batch_create")
        for n in nets:  # the batch keeps its own copy
            n.close()
        self.handle = h
        self.specs = list(specs)
        self.N = np.array([s.n_species for s in specs], np.int64)
        self.M = np.array([s.n_reactions for s in specs], np.int64)
        self.xoff = np.concatenate([[0], np.cumsum(self.N)[:-1]])
        self.moff = np.concatenate([[0], np.cumsum(self.M)[:-1]])
        self.policy = (thread_max_m, warp_max_m, block_threads, blocks_per_sm)

    def info(self):
        ts, tr = ctypes.c_int64(), ctypes.c_int64()
        c = [ctypes.c_int32() for _ in range(3)]
        L.check(self.lib.rt_batch_info(self.handle, ctypes.byref(ts), ctypes.byref(tr), *[ctypes.byref(x) for x in c]),
                "rt_batch_info")
        return dict(total_species=ts.value, total_reactions=tr.value, n_thread=c[0].value, n_warp=c[1].value,
                    n_block=c[2].value)

    def outputs(self, n_traj: int, grad: bool = False, trace_len: int = 0):
        """Device tensors for a run: x_final packed [net i][traj j][N_i]; n_events, status, t_last
        [n_nets, n_traj]; with grad also loglik [n_nets, n_traj] and counts / t_internal packed
        [net i][traj j][M_i]; with trace_len also trace_mu / trace_t [n_nets, n_traj, trace_len]."""
        dev = torch.device("cuda", torch.cuda.current_device())
        n = len(self.specs)
        out = dict(x_final=torch.empty(int(self.N.sum()) * n_traj, dtype=torch.int32, device=dev),
                   n_events=torch.empty((n, n_traj), dtype=torch.int64, device=dev),
                   status=torch.empty((n, n_traj), dtype=torch.int32, device=dev),
                   t_last=torch.empty((n, n_traj), dtype=torch.float64, device=dev))
        if grad:
            out["loglik"] = torch.empty((n, n_traj), dtype=torch.float64, device=dev)
            out["counts"] = torch.empty(int(self.M.sum()) * n_traj, dtype=torch.int32, device=dev)
            out["t_internal"] = torch.empty(int(self.M.sum()) * n_traj, dtype=torch.float64, device=dev)
        if trace_len:
            out["trace_mu"] = torch.empty((n, n_traj, int(trace_len)), dtype=torch.int32, device=dev)
            out["trace_t"] = torch.empty((n, n_traj, int(trace_len)), dtype=torch.float64, device=dev)
        return out

    def run(self, x0: torch.Tensor, t_end: torch.Tensor, n_traj: int, seed: int = 1,
            max_events: int = (1 << 31) - 1, outputs: Optional[dict] = None) -> dict:
        """x0: packed int32 device tensor (sum of N_i); t_end: float64 device tensor [n_nets]."""
        out = outputs if outputs is not None else self.outputs(n_traj)
        o = L.rt_batch_outputs()
        o.x_final_dev = _ptr(out.get("x_final"))
        o.n_events_dev = _ptr(out.get("n_events"))
        o.status_dev = _ptr(out.get("status"))
        o.t_last_dev = _ptr(out.get("t_last"))
        o.loglik_dev = _ptr(out.get("loglik"))
        o.counts_dev = _ptr(out.get("counts"))
        o.t_internal_dev = _ptr(out.get("t_internal"))
        if "trace_mu" in out:
            o.trace_len = int(out["trace_mu"].shape[2])
            o.trace_mu_dev = _ptr(out["trace_mu"])
            o.trace_t_dev = _ptr(out.get("trace_t"))
        L.check(self.lib.rt_batch_run(self.handle, _ptr(x0), _ptr(t_end), int(max_events), int(seed) & (2**64 - 1),
                                      int(n_traj), ctypes.byref(o), _stream()), "rt_batch_run")
        return out

    def x_final_of(self, out: dict, i: int, n_traj: int) -> torch.Tensor:
        """[n_traj, N_i] final states of network i from the packed output."""
        b = int(self.xoff[i]) * n_traj
        return out["x_final"][b:b + n_traj * int(self.N[i])].view(n_traj, int(self.N[i]))

    def per_channel_of(self, out: dict, key: str, i: int, n_traj: int) -> torch.Tensor:
        """[n_traj, M_i] counts or t_internal of network i from the packed output."""
        b = int(self.moff[i]) * n_traj
        return out[key][b:b + n_traj * int(self.M[i])].view(n_traj, int(self.M[i]))

    def capture(self, x0: torch.Tensor, t_end: torch.Tensor, n_traj: int, seed: int = 1,
                max_events: int = (1 << 31) - 1, grad: bool = False, trace_len: int = 0):
        """Capture one rt_batch_run in a CUDA graph; returns (graph, outputs).  graph.replay() reruns it."""
        out = self.outputs(n_traj, grad=grad, trace_len=trace_len)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(x0, t_end, n_traj, seed, max_events, out)  # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(x0, t_end, n_traj, seed, max_events, out)
        return g, out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def draw_exp1(seed: int, traj, channel, index, stream_id: int = 0):
    """(u, E) of the library's Philox Exp(1) draws for the given (traj, channel, index) triples."""
    lib = L.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    tr = torch.as_tensor(np.asarray(traj, dtype=np.uint64).view(np.int64)).to(dev)
    ch = torch.as_tensor(np.asarray(channel, dtype=np.uint32).view(np.int32)).to(dev)
    ix = torch.as_tensor(np.asarray(index, dtype=np.uint64).view(np.int64)).to(dev)
    n = tr.numel()
    u = torch.empty(n, dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    L.check(lib.rt_draw_exp1(int(seed), int(stream_id), n, _ptr(tr), _ptr(ch), _ptr(ix), _ptr(u), _ptr(e),
                             _stream()), "rt_draw_exp1")
    return u, e


def log_eval(x: torch.Tensor) -> torch.Tensor:
    lib = L.load()
    x = x.to(torch.float64).contiguous()
    y = torch.empty_like(x)
    L.check(lib.rt_log_eval(x.numel(), _ptr(x), _ptr(y), _stream()), "rt_log_eval")
    return y


def philox(ctr: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    lib = L.load()
    c = ctr.contiguous()
    out = torch.empty_like(c)
    L.check(lib.rt_philox(c.numel() // 4, _ptr(c), int(key0), int(key1), _ptr(out), _stream()), "rt_philox")
    return out


def fp64_probe(iters: int = 4096, blocks_per_sm: int = 8, repeats: int = 3):
    """Measured binary64 add/multiply issue rate (operations per second) of the current GPU:
    the best of `repeats` timed rt_fp64_probe launches (CUDA events on the current stream)."""
    lib = L.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    ops = ctypes.c_double(0.0)
    stream = torch.cuda.current_stream()
    L.check(lib.rt_fp64_probe(int(iters), int(blocks_per_sm), _ptr(sink), ctypes.byref(ops), _stream()),
            "rt_fp64_probe")  # warm-up
    best = 0.0
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        L.check(lib.rt_fp64_probe(int(iters), int(blocks_per_sm), _ptr(sink), ctypes.byref(ops), _stream()),
                "rt_fp64_probe")
        b.record(stream)
        b.synchronize()
        best = max(best, ops.value / (a.elapsed_time(b) / 1e3))
    return best


def parse_model(text: str):
    """Parse a model in the text format of the paper's Table 4 (rt_model_parse).  Returns a dict:
    net (a workloads.Network), x0 (int32 [N]), names, time (None if absent), steps (None if absent)."""
    lib = L.load()
    p = ctypes.POINTER(L.rt_model)()
    L.check(lib.rt_model_parse(text.encode(), ctypes.byref(p)), "rt_model_parse")
    try:
        m = p.contents
        N, M = m.n_species, m.n_reactions

        def arr(ptr, n, dt):
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt).copy() if n else np.zeros(0, dt)

        net = NetworkSpec(N, M, arr(m.reac_rxn, m.n_reac_nz, np.int32), arr(m.reac_sp, m.n_reac_nz, np.int32),
                          arr(m.reac_coef, m.n_reac_nz, np.int32), arr(m.stoi_rxn, m.n_stoi_nz, np.int32),
                          arr(m.stoi_sp, m.n_stoi_nz, np.int32), arr(m.stoi_delta, m.n_stoi_nz, np.int32),
                          arr(m.c, M, np.float64), "model")
        names = [m.species_names[i].decode() for i in range(N)]
        return dict(net=net, x0=arr(m.x0, N, np.int32), names=names,
                    time=None if math.isnan(m.time) else float(m.time), steps=None if m.steps < 0 else int(m.steps))
    finally:
        lib.rt_model_free(p)
