"""The absolute-time form (absolute firing times with the dependency graph, Sec. 5) on the tree
mapping -- a thread-block cluster per trajectory, min-tree argmin, only the touched channels
updated per event -- against the oracle's absolute-time mode, bit for bit, through the C ABI."""
import math
import os

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

ABS = dict(form=L.RT_FORM_ABSOLUTE)
LAZY = dict(mode=oracle.MODE_LAZY)


@pytest.fixture(scope="module")
def mid():
    net = W.random_mass_action(300, 5000, seed=4242, c_sigma=1.0)
    x0 = W.poisson_x0(300, 60, 4243)
    return net, x0


@pytest.mark.parametrize("C", [1, 2, 4, 8, 0])
def test_tree_bit_exact_for_any_cluster_size(mid, C):
    """5000 channels, 5 trajectories, 2000 events each (t_end = inf): every output and the event
    trace bit-identical to the oracle's absolute-time mode, whatever the cluster size."""
    net, x0 = mid
    netg = api.Network(net)
    g = api.simulate(netg, x0, math.inf, 5, seed=9, max_events=2000, grad=True, ctas_per_traj=C, trace_len=2000,
                     **ABS)
    o = oracle.run(net, x0, math.inf, 5, seed=9, max_events=2000, want_grad=True, trace_len=2000, n_threads=5, **LAZY)
    assert (o["status"] == oracle.ST_MAX_EVENTS).all()
    assert_trace(g, o)
    assert_same(g, o)


def test_tree_grid_likelihood_and_per_trajectory_x0_to_finite_horizon(mid):
    net, x0 = mid
    netg = api.Network(net)
    x0m = np.stack([x0, np.roll(x0, 1), x0 // 2]).astype(np.int32)
    g = api.simulate(netg, x0m, 0.002, 3, seed=2, stream_id=3, traj_offset=77, grad=True, grid="traj",
                     sample_dt=0.0001, ctas_per_traj=4, trace_len=500, **ABS)
    o = oracle.run(net, x0m, 0.002, 3, seed=2, stream_id=3, traj_offset=77, want_grad=True, want_grid=True,
                   sample_dt=0.0001, trace_len=500, n_threads=3, **LAZY)
    assert (o["status"] == oracle.ST_TEND).all() and (o["n_events"] > 100).all()
    assert_trace(g, o)
    assert_same(g, o)


def test_tree_small_networks_absorption_bad_x0_and_dimers():
    """Networks of a few dozen channels (one group), absorption, a negative initial count, 2A
    reactions (one reader entry per distinct species) and channels reading two changed species."""
    for seed in range(4):
        net = W.random_mass_action(3, 40 + 17 * seed, seed=seed + 70)
        x0 = W.poisson_x0(3, 15, seed)
        g = api.simulate(api.Network(net), x0, 5.0, 7, seed=seed, grad=True, max_events=5000, trace_len=300, **ABS)
        o = oracle.run(net, x0, 5.0, 7, seed=seed, want_grad=True, max_events=5000, trace_len=300, n_threads=7,
                       **LAZY)
        assert_trace(g, o)
        assert_same(g, o)
    death = W._from_lists(2, [({0: 1}, {}, 1.0), ({1: 1}, {}, 2.0)] * 20, "death40")
    x0 = np.array([[3, 4], [-1, 2]], np.int32)
    g = api.simulate(api.Network(death), x0, 100.0, 2, seed=1, grad=True, **ABS)
    o = oracle.run(death, x0, 100.0, 2, seed=1, want_grad=True, **LAZY)
    assert o["status"].tolist() == [oracle.ST_ABSORBED, oracle.ST_BAD_X0]
    assert_same(g, o)


def test_tree_overflow_stops_before_the_event():
    birth = W.pure_birth(1e6)
    g = api.simulate(api.Network(birth), [2**31 - 3], math.inf, 2, seed=1, grad=True, **ABS)
    o = oracle.run(birth, [2**31 - 3], math.inf, 2, seed=1, want_grad=True, **LAZY)
    assert (o["status"] == oracle.ST_OVERFLOW).all()
    assert_same(g, o)


def test_tree_form_and_mapping_must_match(mid):
    net, x0 = mid
    netg = api.Network(net)
    with pytest.raises(L.RandtimeError):
        api.simulate(netg, x0, 1.0, 1, mapping=L.RT_MAP_TREE)
    with pytest.raises(L.RandtimeError):
        api.simulate(netg, x0, 1.0, 1, mapping=L.RT_MAP_BUNDLE, **ABS)


def test_tree_bounded_wait_reports_timeout_without_hanging(mid):
    """A mailbox poll limit of zero makes the CTAs of a cluster give up waiting for each other:
    status TIMEOUT, no hang, and the context stays usable."""
    net, x0 = mid
    netg = api.Network(net)
    old = os.environ.get("RT_DEBUG_SPIN_LIMIT")
    os.environ["RT_DEBUG_SPIN_LIMIT"] = "0"
    try:
        g = api.simulate(netg, x0, math.inf, 3, seed=1, max_events=2000, ctas_per_traj=8, **ABS)
        torch.cuda.synchronize()
    finally:
        if old is None:
            del os.environ["RT_DEBUG_SPIN_LIMIT"]
        else:
            os.environ["RT_DEBUG_SPIN_LIMIT"] = old
    assert (g["status"].cpu().numpy() == L.RT_TRAJ_TIMEOUT).all()
    g2 = api.simulate(netg, x0, math.inf, 1, seed=1, max_events=50, ctas_per_traj=8, **ABS)
    o = oracle.run(net, x0, math.inf, 1, seed=1, max_events=50, **LAZY)
    assert_same(g2, o, keys=("x_final", "n_events", "status", "t_last"))


@pytest.mark.slow
def test_tree_full_size_large_network_event_by_event():
    """N = 1e4, M = 1e6 at the benchmarked launch (16 trajectories, library-chosen cluster size):
    the first 3000 events of two trajectories against the oracle, event by event, with their
    counts, internal times and final states; X = X0 + sum n_k v_k exactly for all 16."""
    cfg = W.large_network_config(max_events=3000)
    net, x0 = cfg["net"], cfg["x0"]
    netg = api.Network(net)
    g = api.simulate(netg, x0, math.inf, 16, seed=1, max_events=3000, grad=True, trace_len=3000, **ABS)
    torch.cuda.synchronize()
    for j in (0, 13):
        o = oracle.run(net, x0, math.inf, 1, seed=1, traj_offset=j, max_events=3000, want_grad=True,
                       trace_len=3000, **LAZY)
        assert_trace(g, o, idx=slice(j, j + 1))
        for k in ("x_final", "n_events", "status", "counts"):
            assert np.array_equal(g[k][j].cpu().numpy(), o[k][0]), k
        for k in ("t_last", "t_internal", "loglik"):
            assert np.array_equal(g[k][j].cpu().numpy().view(np.int64), o[k][0].view(np.int64)), k
    counts = g["counts"].cpu().numpy().astype(np.int64)
    expect = np.tile(x0.astype(np.int64), (16, 1))
    for j in range(16):
        np.add.at(expect[j], net.stoi_sp, counts[j, net.stoi_rxn] * net.stoi_delta)
    assert np.array_equal(g["x_final"].cpu().numpy(), expect)
