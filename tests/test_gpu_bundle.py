"""Large-network mode (several thread blocks per trajectory, state streamed through HBM)
against the CPU oracle, bit for bit, through the C ABI."""
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

B.build()


@pytest.fixture(scope="module")
def mid():
    net = W.random_mass_action(300, 5000, seed=4242, c_sigma=1.0)
    x0 = W.poisson_x0(300, 60, 4243)
    return net, x0


@pytest.mark.parametrize("C", [1, 3, 8, 0])
def test_bundle_bit_exact_for_any_block_count(mid, C):
    """5000 channels, 5 trajectories, 2000 events each (t_end = inf): every output bit-identical."""
    net, x0 = mid
    netg = api.Network(net)
    g = api.simulate(netg, x0, math.inf, 5, seed=9, max_events=2000, grad=True, mapping=L.RT_MAP_BUNDLE,
                     ctas_per_traj=C)
    o = oracle.run(net, x0, math.inf, 5, seed=9, max_events=2000, want_grad=True, n_threads=5)
    assert (o["status"] == oracle.ST_MAX_EVENTS).all()
    assert_same(g, o)


def test_bundle_grid_and_likelihood_to_finite_horizon(mid):
    net, x0 = mid
    netg = api.Network(net)
    x0m = np.stack([x0, np.roll(x0, 1), x0 // 2]).astype(np.int32)
    g = api.simulate(netg, x0m, 0.002, 3, seed=2, stream_id=3, traj_offset=77, grad=True, grid="traj",
                     sample_dt=0.0001, mapping=L.RT_MAP_BUNDLE, ctas_per_traj=5)
    o = oracle.run(net, x0m, 0.002, 3, seed=2, stream_id=3, traj_offset=77, want_grad=True, want_grid=True,
                   sample_dt=0.0001, n_threads=3)
    assert (o["status"] == oracle.ST_TEND).all() and (o["n_events"] > 100).all()
    assert_same(g, o)


@pytest.mark.parametrize("n_species", [20000, 40000, 48000])
def test_bundle_copy_ring_depths_fall_back_with_many_species(n_species):
    """Each block mirrors X in shared memory, so many species leave less room for the copy
    ring: 20000 species keep 4 stages, 40000 leave 2 and 48000 one (no copy in flight while a
    pair is processed).  Every depth gives the same bits, for 1 and 8 blocks per trajectory."""
    net = W.random_mass_action(n_species, 3000, seed=515, c_sigma=1.0)
    x0 = W.poisson_x0(n_species, 40, 516)
    o = oracle.run(net, x0, math.inf, 2, seed=4, max_events=300, want_grad=True, n_threads=2)
    for C in (1, 8):
        g = api.simulate(api.Network(net), x0, math.inf, 2, seed=4, max_events=300, grad=True,
                         mapping=L.RT_MAP_BUNDLE, ctas_per_traj=C)
        assert_same(g, o)


def test_bundle_small_networks_and_edge_cases():
    """Networks smaller than a block, absorption and bad initial states in the bundle kernel."""
    for seed in range(3):
        net = W.random_mass_action(3, 40 + seed, seed=seed + 70)
        x0 = W.poisson_x0(3, 15, seed)
        g = api.simulate(api.Network(net), x0, 5.0, 7, seed=seed, grad=True, max_events=5000,
                         mapping=L.RT_MAP_BUNDLE, ctas_per_traj=2)
        o = oracle.run(net, x0, 5.0, 7, seed=seed, want_grad=True, max_events=5000, n_threads=7)
        assert_same(g, o)
    death = W._from_lists(2, [({0: 1}, {}, 1.0), ({1: 1}, {}, 2.0)] * 20, "death40")
    x0 = np.array([[3, 4], [-1, 2]], np.int32)
    g = api.simulate(api.Network(death), x0, 100.0, 2, seed=1, grad=True, mapping=L.RT_MAP_BUNDLE,
                     ctas_per_traj=2)
    o = oracle.run(death, x0, 100.0, 2, seed=1, want_grad=True)
    assert o["status"].tolist() == [oracle.ST_ABSORBED, oracle.ST_BAD_X0]
    assert_same(g, o)


def test_large_network_full_size_first_events_and_invariant():
    """N = 10^4, M = 10^6, 16 trajectories in the benchmarked launch: the first 300 events of two
    trajectories bit-exact against the oracle; X = X0 + sum n_k v_k exactly for all 16."""
    cfg = W.large_network_config()
    net, x0 = cfg["net"], cfg["x0"]
    netg = api.Network(net)
    g = api.simulate(netg, x0, math.inf, 16, seed=1, max_events=300, grad=True, mapping=L.RT_MAP_BUNDLE)
    torch.cuda.synchronize()
    for j in (0, 11):
        o = oracle.run(net, x0, math.inf, 1, seed=1, traj_offset=j, max_events=300, want_grad=True)
        for k in ("x_final", "n_events", "status", "counts"):
            assert np.array_equal(g[k][j].cpu().numpy(), o[k][0]), k
        for k in ("t_last", "t_internal", "loglik"):
            assert np.array_equal(g[k][j].cpu().numpy().view(np.int64), o[k][0].view(np.int64)), k
    counts = g["counts"].cpu().numpy().astype(np.int64)
    expect = np.tile(x0.astype(np.int64), (16, 1))
    for j in range(16):  # sparse X0 + sum_k n_k v_k
        np.add.at(expect[j], net.stoi_sp, counts[j, net.stoi_rxn] * net.stoi_delta)
    assert np.array_equal(g["x_final"].cpu().numpy(), expect)
    assert (g["n_events"].cpu().numpy() == 300).all()


def test_bounded_wait_reports_timeout_without_hanging(mid):
    """A wait limit of zero polls makes the cross-block barrier give up: status TIMEOUT, no hang."""
    net, x0 = mid
    netg = api.Network(net)
    old = os.environ.get("RT_DEBUG_SPIN_LIMIT")
    os.environ["RT_DEBUG_SPIN_LIMIT"] = "0"
    try:
        g = api.simulate(netg, x0, math.inf, 3, seed=1, max_events=2000, mapping=L.RT_MAP_BUNDLE, ctas_per_traj=8)
        torch.cuda.synchronize()
    finally:
        if old is None:
            del os.environ["RT_DEBUG_SPIN_LIMIT"]
        else:
            os.environ["RT_DEBUG_SPIN_LIMIT"] = old
    assert (g["status"].cpu().numpy() == L.RT_TRAJ_TIMEOUT).all()
    # the context is still usable
    g2 = api.simulate(netg, x0, math.inf, 1, seed=1, max_events=50, mapping=L.RT_MAP_BUNDLE, ctas_per_traj=8)
    o = oracle.run(net, x0, math.inf, 1, seed=1, max_events=50)
    assert_same(g2, o, keys=("x_final", "n_events", "status", "t_last"))
