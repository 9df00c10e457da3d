"""The allocation-free large-network entry point, rt_run_bundle_noalloc, against rt_run.

Some callers cannot call cudaMalloc where they simulate: a host application whose
device memory belongs to its own pool allocator, or a latency-critical loop that must
stay out of the driver's allocator.  rt_run_bundle_noalloc runs the bundle kernels with
their scratch in a fixed 16 MiB array inside the library instead of a caller-allocated
workspace.  These tests call it through the C ABI and compare it with rt_run (bundle
mapping, caller workspace) on two calls in a row, bit for bit, and check that a run
needing more scratch than the array holds is refused with an error.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_00405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import _lib as L  # noqa: E402
from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

B.build()

KEYS = ("x_final", "n_events", "status", "t_last", "loglik", "counts", "t_internal")


def _noalloc_run(net, x0, n_traj, seed, offset, max_events, ctas):
    lib = L.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    N, M = net.N, net.M
    out = dict(x_final=torch.empty((n_traj, N), dtype=torch.int32, device=dev),
               n_events=torch.empty(n_traj, dtype=torch.int64, device=dev),
               status=torch.empty(n_traj, dtype=torch.int32, device=dev),
               t_last=torch.empty(n_traj, dtype=torch.float64, device=dev),
               loglik=torch.empty(n_traj, dtype=torch.float64, device=dev),
               counts=torch.empty((n_traj, M), dtype=torch.int32, device=dev),
               t_internal=torch.empty((n_traj, M), dtype=torch.float64, device=dev))
    x0d = torch.as_tensor(x0, dtype=torch.int32).to(dev).contiguous()
    p = L.rt_run_params(ctypes.c_void_p(x0d.data_ptr()), 0, 0, math.inf, max_events, seed, n_traj, offset, 0.0)
    o = L.rt_outputs()
    o.x_final_dev = out["x_final"].data_ptr()
    o.n_events_dev = out["n_events"].data_ptr()
    o.status_dev = out["status"].data_ptr()
    o.t_last_dev = out["t_last"].data_ptr()
    o.loglik_dev = out["loglik"].data_ptr()
    o.counts_dev = out["counts"].data_ptr()
    o.t_internal_dev = out["t_internal"].data_ptr()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.rt_run_bundle_noalloc(net.handle, ctypes.byref(p), ctypes.byref(o), ctas, stream)
    return rc, out, x0d


def test_noalloc_entry_point_matches_rt_run_on_two_calls_in_a_row():
    spec = W.random_mass_action(300, 5000, seed=4242, c_sigma=1.0)
    x0 = W.poisson_x0(300, 60, 4243)
    net = api.Network(spec)
    for seed, offset in ((9, 0), (10, 77)):
        ref = api.simulate(net, x0, math.inf, 5, seed=seed, traj_offset=offset, max_events=2000, grad=True,
                           mapping=L.RT_MAP_BUNDLE, ctas_per_traj=4)
        rc, out, _ = _noalloc_run(net, x0, 5, seed, offset, 2000, 4)
        assert rc == L.RT_OK, L.load().rt_last_error()
        torch.cuda.synchronize()
        assert (out["status"] == L.RT_TRAJ_MAX_EVENTS).all()
        for k in KEYS:
            a, b = out[k].cpu().numpy(), ref[k].cpu().numpy()
            if a.dtype == np.float64:
                assert np.array_equal(a.view(np.int64), b.view(np.int64)), k
            else:
                assert np.array_equal(a, b), k


def test_noalloc_entry_point_refuses_runs_larger_than_its_array():
    spec = W.random_mass_action(300, 5000, seed=4242, c_sigma=1.0)
    net = api.Network(spec)
    rc, _, _ = _noalloc_run(net, W.poisson_x0(300, 60, 4243), 200, 1, 0, 10, 0)  # ~28 MB of scratch
    assert rc == L.RT_ERR_OOM
    assert b"scratch" in L.load().rt_last_error()
