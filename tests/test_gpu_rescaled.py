"""Table 3's form of the method (relative waiting times rescaled by p_k / a_k after every event,
every propensity recomputed; RT_FORM_RESCALED on the thread mapping up to 8 reactions and on a warp
per trajectory up to 256) against the oracle's mode 2, bit for bit, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_00405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import _lib as L  # noqa: E402
from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

from test_gpu_parity import assert_same  # noqa: E402
from test_gpu_trace import assert_trace  # noqa: E402

B.build()

RES = dict(form=L.RT_FORM_RESCALED)
MODE = dict(mode=oracle.MODE_RESCALED)

CASES = {
    "lotka_volterra": (W.lotka_volterra(), np.array([1000, 1000], np.int32), 1.0),
    "birth_death": (W.birth_death(), np.array([0], np.int32), 10.0),
    "dimerisation": (W.dimerisation(), np.array([1000, 0], np.int32), 5.0),
    "isomerisation_frozen": (W.isomerisation(3.0, 1.0), np.array([1, 0], np.int32), 20.0),
    "random_8": (W.random_mass_action(6, 8, seed=91), None, 0.5),
    "random_5": (W.random_mass_action(4, 5, seed=92), None, 0.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_rescaled_form_bit_exact(name):
    net, x0, t_end = CASES[name]
    if x0 is None:
        x0 = W.poisson_x0(net.n_species, 30, 3)
    n = 200
    netg = api.Network(net)
    g = api.simulate(netg, x0, t_end, n, seed=2, stream_id=1, traj_offset=17, max_events=200000, grad=True,
                     grid="traj", sample_dt=t_end / 20, trace_len=500, **RES)
    o = oracle.run(net, x0, t_end, n, seed=2, stream_id=1, traj_offset=17, max_events=200000, want_grad=True,
                   want_grid=True, sample_dt=t_end / 20, trace_len=500, n_threads=16, **MODE)
    assert_same(g, o)
    assert_trace(g, o)


@pytest.mark.parametrize("M,N", [(9, 4), (33, 10), (64, 16), (150, 40), (256, 64)])
def test_rescaled_form_on_the_warp_mapping_bit_exact(M, N):
    net = W.random_mass_action(N, M, seed=970 + M, c_sigma=0.6)
    x0 = W.poisson_x0(N, 25, M)
    n = 45  # a ragged last block of warps
    t_end = 0.5 if M <= 64 else 0.2
    netg = api.Network(net)
    g = api.simulate(netg, x0, t_end, n, seed=M, stream_id=3, traj_offset=2, max_events=100000, grad=True,
                     grid="traj", sample_dt=t_end / 10, trace_len=300, **RES)
    o = oracle.run(net, x0, t_end, n, seed=M, stream_id=3, traj_offset=2, max_events=100000, want_grad=True,
                   want_grid=True, sample_dt=t_end / 10, trace_len=300, n_threads=16, **MODE)
    assert o["n_events"].mean() > 10
    assert_same(g, o)
    assert_trace(g, o)
    # the warp kernel on a small network too (explicit mapping), with an event cap
    small = W.random_mass_action(4, 5, seed=92)
    xs = W.poisson_x0(4, 30, 3)
    gs = api.simulate(api.Network(small), xs, 0.5, 70, seed=2, max_events=25, grad=True, mapping=L.RT_MAP_WARP,
                      **RES)
    os_ = oracle.run(small, xs, 0.5, 70, seed=2, max_events=25, want_grad=True, n_threads=16, **MODE)
    assert_same(gs, os_)


def test_rescaled_form_moments_and_absorption():
    net, x0 = W.dimerisation(), np.array([1000, 0], np.int32)
    netg = api.Network(net)
    g = api.simulate(netg, x0, 2.0, 3000, seed=5, sample_dt=0.1, grid="moments", **RES)
    o = oracle.run(net, x0, 2.0, 3000, seed=5, sample_dt=0.1, want_grid=True, n_threads=16, **MODE)
    grid = o["grid"].astype(np.int64)
    assert np.array_equal(g["grid_sum"].cpu().numpy(), grid.sum(0))
    assert np.array_equal(g["grid_sumsq"].cpu().numpy(), (grid ** 2).sum(0))
    death = W._from_lists(1, [({0: 1}, {}, 1.0)], "death")
    gd = api.simulate(api.Network(death), np.array([[5], [-1]], np.int32), math.inf, 2, seed=1, grad=True, **RES)
    od = oracle.run(death, np.array([[5], [-1]], np.int32), math.inf, 2, seed=1, want_grad=True, **MODE)
    assert od["status"].tolist() == [oracle.ST_ABSORBED, oracle.ST_BAD_X0]
    assert_same(gd, od)


def test_rescaled_form_limits():
    netg = api.Network(W.random_mass_action(6, 12, seed=93))
    x0 = W.poisson_x0(6, 10, 1)
    with pytest.raises(L.RandtimeError):
        api.simulate(netg, x0, 1.0, 4, mapping=L.RT_MAP_THREAD, **RES)  # M > 8 on the thread mapping
    with pytest.raises(L.RandtimeError):
        api.simulate(netg, x0, 1.0, 4, mapping=L.RT_MAP_BLOCK, **RES)
    with pytest.raises(L.RandtimeError):
        api.simulate(netg, x0, 1.0, 4, mapping=L.RT_MAP_WARP, lanes_per_traj=8, **RES)
    big = api.Network(W.random_mass_action(60, 300, seed=94))
    with pytest.raises(L.RandtimeError):
        api.simulate(big, W.poisson_x0(60, 10, 1), 1.0, 4, **RES)  # M > 256


def test_table3_workload_at_full_size_sampled():
    """The benchmarked launches of Table 3's form: 2^18 Lotka-Volterra trajectories to t_end = 10 on
    the thread mapping, and 16384 trajectories of the M = 64 gradient network to t_end = 5 on the warp
    mapping; sampled trajectories against the oracle, bit for bit (the oracle re-runs each sampled
    trajectory alone by its global id)."""
    cfg = W.ensemble_configs(1 << 18)[0]
    g = api.simulate(api.Network(cfg["net"]), cfg["x0"], cfg["t_end"], 1 << 18, seed=1, max_events=cfg["max_events"],
                     mapping=L.RT_MAP_THREAD, **RES)
    torch.cuda.synchronize()
    for j in (0, 1, 4097, 100000, (1 << 18) - 1):
        o = oracle.run(cfg["net"], cfg["x0"], cfg["t_end"], 1, seed=1, traj_offset=j, max_events=cfg["max_events"],
                       **MODE)
        assert_same(g, o, keys=("x_final", "n_events", "status", "t_last"), idx=slice(j, j + 1))
    gc = W.grad_config(16384)
    gg = api.simulate(api.Network(gc["net"]), gc["x0"], gc["t_end"], 16384, seed=1, max_events=10**8,
                      mapping=L.RT_MAP_WARP, **RES)
    torch.cuda.synchronize()
    for j in (0, 31, 8191, 16383):
        o = oracle.run(gc["net"], gc["x0"], gc["t_end"], 1, seed=1, traj_offset=j, max_events=10**8, **MODE)
        assert_same(gg, o, keys=("x_final", "n_events", "status", "t_last"), idx=slice(j, j + 1))
