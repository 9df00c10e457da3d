"""CPU oracle for the next reaction random time algorithm (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
``oracle.c`` is a plain single-trajectory loop compiled with gcc
(``-O2 -ffp-contract=off``, no fast-math), and this file only marshals numpy
arrays into it.

Functions (all follow Liu & Wang, arXiv:2103.00405):
  philox4x32_10  -- Philox4x32-10 block function (Salmon et al., SC'11)
  rt_log         -- fixed-point natural log rounded once to binary64
  exp1 / uniform -- the Exp(1) internal-time increment of Eq. 24 and its uniform
  grid_len       -- number of sampling points on [0, t_end]
  run            -- the NRRTA loop of Table 2 (Eq. 24-27) for many trajectories, in the
                    internal-time form or the absolute-time (dependency graph) form
  loglik_backward-- d(sum_j w_j l_j)/dc from saved counts and internal times
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-std=gnu11"]

ST_TEND, ST_MAX_EVENTS, ST_ABSORBED, ST_OVERFLOW, ST_TIMEOUT, ST_BAD_X0 = 0, 1, 2, 3, 4, 5


def build(force: bool = False, out: str = _LIB, extra_flags=()) -> str:
    """Compile oracle.c into a shared library (gcc)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, *extra_flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def _declare(lib):
    i32, i64, u32, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_rt_log.argtypes = [dbl]
    lib.oracle_rt_log.restype = dbl
    lib.oracle_exp1.argtypes = [u64, u64, u32, u64, u32]
    lib.oracle_exp1.restype = dbl
    lib.oracle_uniform.argtypes = [u64, u64, u32, u64, u32]
    lib.oracle_uniform.restype = dbl
    lib.oracle_grid_len.argtypes = [dbl, dbl]
    lib.oracle_grid_len.restype = i64
    lib.oracle_run.argtypes = [i32, i32, i32, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32,
                               dbl, i64, u64, u32, i64, i64, dbl,
                               vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, i32]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_loglik_backward.argtypes = [i32, i64, vp, vp, vp, vp, vp]
    lib.oracle_loglik_backward.restype = None
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  A custom path loads a variant build."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            # ORACLE_LIB points the pins at a variant build (the mutation test uses it)
            _lib = _declare(ctypes.CDLL(os.environ.get("ORACLE_LIB") or build()))
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key, lib=None) -> np.ndarray:
    lib = lib or load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def rt_log(x: float, lib=None) -> float:
    return (lib or load()).oracle_rt_log(float(x))


def exp1(seed, traj, k, n, stream=0, lib=None) -> float:
    return (lib or load()).oracle_exp1(seed, traj, k, n, stream)


def uniform(seed, traj, k, n, stream=0, lib=None) -> float:
    return (lib or load()).oracle_uniform(seed, traj, k, n, stream)


def grid_len(t_end: float, sample_dt: float, lib=None) -> int:
    return int((lib or load()).oracle_grid_len(float(t_end), float(sample_dt)))


MODE_EAGER, MODE_LAZY, MODE_RESCALED = 0, 1, 2


def run(net, x0, t_end, n_traj, seed=1, stream_id=0, traj_offset=0, max_events=(1 << 31) - 1,
        sample_dt=0.0, want_grid=False, want_grad=False, trace_len=0, n_threads=1, lib=None,
        mode=MODE_EAGER, enabled=None, beta=None):
    """Run the oracle; returns a dict of numpy arrays.

    x0 is [N] (shared) or [n_traj, N] (per trajectory).  mode: MODE_EAGER (Table 2 in
    internal-time form), MODE_LAZY (absolute-time form with the dependency graph) or
    MODE_RESCALED (Table 3's rescaled waiting times, every propensity recomputed).
    enabled: optional [M] flags; channels with 0 never fire (frozen internal time).
    beta: optional [M] rate slopes, c_k(t) = c_k (1 + beta_k t), beta_k >= 0 (mode 0 only).
    """
    lib = lib or load()
    N, M = int(net.n_species), int(net.n_reactions)
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    per = 1 if x0.ndim == 2 else 0
    n_traj = int(n_traj)
    G = lib.oracle_grid_len(float(t_end), float(sample_dt)) if want_grid else 0
    out = dict(
        x_final=np.zeros((n_traj, N), np.int32),
        n_events=np.zeros(n_traj, np.int64),
        status=np.zeros(n_traj, np.int32),
        t_last=np.zeros(n_traj, np.float64),
    )
    if want_grid:
        out["grid"] = np.zeros((n_traj, G, N), np.int32)
    if want_grad:
        out["loglik"] = np.zeros(n_traj, np.float64)
        out["counts"] = np.zeros((n_traj, M), np.int32)
        out["t_internal"] = np.zeros((n_traj, M), np.float64)
    if trace_len:
        out["trace_mu"] = np.zeros((n_traj, trace_len), np.int32)
        out["trace_t"] = np.zeros((n_traj, trace_len), np.float64)
    en = None if enabled is None else np.ascontiguousarray(enabled, dtype=np.uint8)
    if en is not None and en.shape != (M,):
        raise ValueError("enabled must have one entry per reaction")
    bt = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    if bt is not None and bt.shape != (M,):
        raise ValueError("beta must have one entry per reaction")
    rc = lib.oracle_run(int(mode), N, M, len(net.reac_rxn), _p(net.reac_rxn), _p(net.reac_sp), _p(net.reac_coef),
                        len(net.stoi_rxn), _p(net.stoi_rxn), _p(net.stoi_sp), _p(net.stoi_delta),
                        _p(net.c), _p(en), _p(bt), _p(x0), per, float(t_end), int(max_events), int(seed), int(stream_id),
                        n_traj, int(traj_offset), float(sample_dt),
                        _p(out["x_final"]), _p(out.get("grid")), _p(out["n_events"]), _p(out["status"]),
                        _p(out["t_last"]), _p(out.get("loglik")), _p(out.get("counts")),
                        _p(out.get("t_internal")), int(trace_len), _p(out.get("trace_mu")),
                        _p(out.get("trace_t")), int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_run failed with %d" % rc)
    return out


def loglik_backward(grad_ll, counts, t_internal, c, lib=None) -> np.ndarray:
    lib = lib or load()
    g = np.ascontiguousarray(grad_ll, dtype=np.float64)
    n = np.ascontiguousarray(counts, dtype=np.int32)
    T = np.ascontiguousarray(t_internal, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    M = n.shape[1]
    out = np.zeros(M, np.float64)
    lib.oracle_loglik_backward(M, n.shape[0], _p(g), _p(n), _p(T), _p(c), _p(out))
    return out
