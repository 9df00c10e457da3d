"""ctypes binding of librandtime (include/randtime.h): argument marshalling only.

Every function here has the C name and signature of the entry point it wraps.
The library is loaded from this package directory; if it is missing the import
fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librandtime.so")

i32, u32, i64, u64, dbl, vp, sz = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)

RT_OK, RT_ERR_INVALID_ARG, RT_ERR_UNSUPPORTED, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
RT_TRAJ_TEND, RT_TRAJ_MAX_EVENTS, RT_TRAJ_ABSORBED, RT_TRAJ_OVERFLOW, RT_TRAJ_TIMEOUT, RT_TRAJ_BAD_X0 = range(6)
RT_MAP_AUTO, RT_MAP_THREAD, RT_MAP_WARP, RT_MAP_BLOCK, RT_MAP_BUNDLE, RT_MAP_TREE = -1, 0, 1, 2, 3, 4
RT_FORM_INTERNAL, RT_FORM_ABSOLUTE, RT_FORM_RESCALED = 0, 1, 2


class rt_launch_cfg(ctypes.Structure):
    _fields_ = [("mapping", i32), ("block_threads", i32), ("ctas_per_traj", i32), ("lanes_per_traj", i32)]


class rt_run_params(ctypes.Structure):
    _fields_ = [("x0_dev", vp), ("per_traj_x0", i32), ("stream_id", u32), ("t_end", dbl), ("max_events", i64),
                ("seed", u64), ("n_traj", i64), ("traj_offset", i64), ("sample_dt", dbl), ("form", i32),
                ("reserved", i32)]


class rt_batch_policy(ctypes.Structure):
    _fields_ = [("thread_max_m", i32), ("warp_max_m", i32), ("block_threads", i32), ("blocks_per_sm", i32)]


class rt_outputs(ctypes.Structure):
    _fields_ = [("x_final_dev", vp), ("grid_dev", vp), ("grid_sum_dev", vp), ("grid_sumsq_dev", vp),
                ("grid_count_dev", vp), ("n_events_dev", vp), ("status_dev", vp), ("t_last_dev", vp),
                ("loglik_dev", vp), ("counts_dev", vp), ("t_internal_dev", vp), ("trace_len", i64),
                ("trace_mu_dev", vp), ("trace_t_dev", vp)]


class rt_batch_outputs(ctypes.Structure):
    _fields_ = [("x_final_dev", vp), ("n_events_dev", vp), ("status_dev", vp), ("t_last_dev", vp),
                ("loglik_dev", vp), ("counts_dev", vp), ("t_internal_dev", vp), ("trace_len", i64),
                ("trace_mu_dev", vp), ("trace_t_dev", vp)]


class rt_model(ctypes.Structure):
    _fields_ = [("n_species", i32), ("n_reactions", i32), ("n_reac_nz", i64), ("reac_rxn", ctypes.POINTER(i32)),
                ("reac_sp", ctypes.POINTER(i32)), ("reac_coef", ctypes.POINTER(i32)), ("n_stoi_nz", i64),
                ("stoi_rxn", ctypes.POINTER(i32)), ("stoi_sp", ctypes.POINTER(i32)), ("stoi_delta", ctypes.POINTER(i32)),
                ("c", ctypes.POINTER(dbl)), ("x0", ctypes.POINTER(i32)), ("species_names", ctypes.POINTER(ctypes.c_char_p)),
                ("time", dbl), ("steps", i64)]


# (name, restype, argtypes) of every entry point declared in include/randtime.h
SIGNATURES = [
    ("rt_network_create", ctypes.c_int, [i32, i32, i64, vp, vp, vp, i64, vp, vp, vp, vp, ctypes.POINTER(vp)]),
    ("rt_network_destroy", None, [vp]),
    ("rt_network_info", ctypes.c_int, [vp, vp, vp, vp, vp]),
    ("rt_network_set_enabled", ctypes.c_int, [vp, vp]),
    ("rt_network_set_rate_slopes", ctypes.c_int, [vp, vp]),
    ("rt_model_parse", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.POINTER(rt_model))]),
    ("rt_model_free", None, [ctypes.POINTER(rt_model)]),
    ("rt_grid_len", i64, [dbl, dbl]),
    ("rt_workspace_bytes", ctypes.c_int, [vp, ctypes.POINTER(rt_run_params), ctypes.POINTER(rt_launch_cfg),
                                          ctypes.POINTER(sz)]),
    ("rt_run", ctypes.c_int, [vp, ctypes.POINTER(rt_run_params), ctypes.POINTER(rt_outputs),
                              ctypes.POINTER(rt_launch_cfg), vp, sz, vp]),
    ("rt_run_bundle_noalloc", ctypes.c_int, [vp, ctypes.POINTER(rt_run_params), ctypes.POINTER(rt_outputs), i32,
                                             vp]),
    ("rt_loglik_backward", ctypes.c_int, [vp, i64, vp, vp, vp, vp, vp]),
    ("rt_draw_exp1", ctypes.c_int, [u64, u32, i64, vp, vp, vp, vp, vp, vp]),
    ("rt_log_eval", ctypes.c_int, [i64, vp, vp, vp]),
    ("rt_philox", ctypes.c_int, [i64, vp, u32, u32, vp, vp]),
    ("rt_batch_create", ctypes.c_int, [i32, vp, vp, ctypes.POINTER(rt_batch_policy), ctypes.POINTER(vp)]),
    ("rt_batch_destroy", None, [vp]),
    ("rt_batch_info", ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
    ("rt_batch_run", ctypes.c_int, [vp, vp, vp, i64, u64, i64, ctypes.POINTER(rt_batch_outputs), vp]),
    ("rt_fp64_probe", ctypes.c_int, [i64, i32, vp, ctypes.POINTER(dbl), vp]),
    ("rt_last_error", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class RandtimeError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed (%d): %s" % (where, code, msg))
        self.code = code


def load(path: str | None = None):
    """Load librandtime.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError("librandtime.so not built (run __graft_entry__.build() or "
                              "python -m paper_2103_00405_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(rc: int, where: str):
    if rc != RT_OK:
        raise RandtimeError(rc, where, load().rt_last_error().decode())
    return rc


def declared_symbols(header: str) -> list:
    """Names of the functions include/randtime.h declares (parsed from the header text)."""
    import re
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", txt)))
