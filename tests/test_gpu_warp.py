"""Warp-segment mapping (8, 16 or 32 lanes per trajectory; networks of 17..256 reactions)
against the CPU oracle, bit for bit, including the gradient workload (M = 64, N = 16) and its
backward kernel."""
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


@pytest.mark.parametrize("M,N", [(17, 5), (32, 8), (33, 8), (64, 16), (100, 25), (129, 30), (256, 64)])
def test_warp_mapping_bit_exact(M, N):
    net = W.random_mass_action(N, M, seed=500 + M, c_sigma=0.7)
    rng = np.random.default_rng(M)
    x0 = rng.integers(0, 30, size=(45, N)).astype(np.int32)
    netg = api.Network(net)
    g = api.simulate(netg, x0, 0.5, 45, seed=M, stream_id=2, traj_offset=5, max_events=30000, sample_dt=0.05,
                     grid="traj", grad=True, mapping=L.RT_MAP_WARP)
    o = oracle.run(net, x0, 0.5, 45, seed=M, stream_id=2, traj_offset=5, max_events=30000, sample_dt=0.05,
                   want_grid=True, want_grad=True, n_threads=16)
    assert_same(g, o)


@pytest.mark.parametrize("G,M,N", [(8, 17, 5), (8, 29, 7), (8, 64, 16), (16, 40, 9), (16, 100, 25), (16, 128, 30),
                                   (32, 17, 5), (32, 64, 16), (32, 200, 50)])
@pytest.mark.parametrize("n_traj", [1, 7, 45])
def test_warp_segments_bit_exact_for_every_width(G, M, N, n_traj):
    """Several trajectories per warp advance together (4 with 8 lanes each, 2 with 16); trajectory
    counts that leave a warp partly empty, ragged channel counts, likelihood, grid and trace."""
    net = W.random_mass_action(N, M, seed=700 + M, c_sigma=0.7)
    rng = np.random.default_rng(M + n_traj)
    x0 = rng.integers(0, 30, size=(n_traj, N)).astype(np.int32)
    if n_traj > 3:
        x0[3, 0] = -1  # one trajectory in a shared warp starts from a bad state
    netg = api.Network(net)
    g = api.simulate(netg, x0, 0.4, n_traj, seed=M, stream_id=1, traj_offset=9, max_events=20000, sample_dt=0.05,
                     grid="traj", grad=True, mapping=L.RT_MAP_WARP, lanes_per_traj=G, trace_len=300)
    o = oracle.run(net, x0, 0.4, n_traj, seed=M, stream_id=1, traj_offset=9, max_events=20000, sample_dt=0.05,
                   want_grid=True, want_grad=True, trace_len=300, n_threads=16)
    assert_same(g, o)
    for k in ("trace_mu", "trace_t"):
        a, b = g[k].cpu().numpy(), o[k]
        assert np.array_equal(a.view(np.int64) if a.dtype == np.float64 else a,
                              b.view(np.int64) if b.dtype == np.float64 else b), k


def test_warp_segments_with_uneven_event_counts_and_caps():
    """Trajectories sharing a warp finish at different events (caps, absorption, t_end); the
    others keep going with the finished lanes idle."""
    death = W._from_lists(2, [({0: 1}, {}, 1.0), ({1: 1}, {}, 2.0)] * 12, "death24")
    x0 = np.array([[3, 4], [0, 0], [40, 1], [7, 7], [1, 300], [2, 2], [9, 0]], np.int32)
    for G in (8, 16, 32):
        for cap in (5, 10**6):
            g = api.simulate(api.Network(death), x0, 3.0, 7, seed=2, grad=True, max_events=cap,
                             mapping=L.RT_MAP_WARP, lanes_per_traj=G)
            o = oracle.run(death, x0, 3.0, 7, seed=2, want_grad=True, max_events=cap)
            assert_same(g, o)


def test_warp_mapping_is_the_default_for_mid_size_networks():
    net = W.random_mass_action(10, 40, seed=3)
    lib = L.load()
    netg = api.Network(net)
    g = api.simulate(netg, W.poisson_x0(10, 20, 1), 0.3, 10, seed=1, grad=True)
    o = oracle.run(net, W.poisson_x0(10, 20, 1), 0.3, 10, seed=1, want_grad=True)
    assert_same(g, o)
    assert lib is not None


def test_warp_moments_equal_sums_of_oracle_grids():
    net = W.random_mass_action(6, 24, seed=11, c_sigma=0.5)
    x0 = W.poisson_x0(6, 25, 12)
    netg = api.Network(net)
    g = api.simulate(netg, x0, 1.0, 301, seed=4, sample_dt=0.1, grid="moments", mapping=L.RT_MAP_WARP,
                     max_events=50000)
    o = oracle.run(net, x0, 1.0, 301, seed=4, sample_dt=0.1, want_grid=True, max_events=50000, n_threads=16)
    known = (o["status"] == 0) | (o["status"] == 2)
    grid = o["grid"].astype(np.int64)
    ok = grid >= 0
    assert np.array_equal(g["grid_sum"].cpu().numpy(), np.where(ok, grid, 0).sum(0))
    assert np.array_equal(g["grid_sumsq"].cpu().numpy(), np.where(ok, grid ** 2, 0).sum(0))
    assert np.array_equal(g["grid_count"].cpu().numpy(), ok[:, :, 0].sum(0))
    assert known.sum() > 0


def test_gradient_workload_full_size_sampled():
    """M = 64, N = 16, 65536 trajectories to t_end = 5 (the benchmarked gradient launch): 12 trajectories
    re-run one by one in the oracle, bit for bit; the backward kernel against the closed form."""
    cfg = W.grad_config()
    net, x0, n = cfg["net"], cfg["x0"], cfg["n_traj"]
    c = torch.tensor(net.c, dtype=torch.float64, requires_grad=True)
    ll = api.LogLik.apply(c, net, x0, cfg["t_end"], n, 1, 0, 10**8)
    ll.sum().backward()
    torch.cuda.synchronize()
    llh = ll.detach().cpu().numpy()
    for j in np.linspace(0, n - 1, 12).astype(np.int64):
        o = oracle.run(net, x0, cfg["t_end"], 1, seed=1, traj_offset=int(j), max_events=10**8, want_grad=True)
        assert llh[j].view(np.int64) == o["loglik"][0].view(np.int64) or (np.isnan(llh[j]) and np.isnan(o["loglik"][0]))
    # closed form of the gradient from a fresh forward run's saved counts and internal times
    out = api.simulate(api.Network(net), x0, cfg["t_end"], n, seed=1, max_events=10**8, grad=True)
    counts = out["counts"].cpu().numpy().astype(np.float64)
    T = out["t_internal"].cpu().numpy()
    closed = ((counts - T) / net.c).sum(0)
    scale = np.maximum(np.abs(closed), (counts / net.c).sum(0))
    assert (np.abs(c.grad.numpy() - closed) <= 1e-9 * scale).all()


@pytest.mark.parametrize("M,N,B", [(257, 60, 0), (600, 150, 0), (1500, 300, 256), (4096, 1024, 512)])
def test_block_mapping_bit_exact(M, N, B):
    """One block per trajectory with all channel state in registers (up to 8 channels per thread)."""
    net = W.random_mass_action(N, M, seed=900 + M, c_sigma=0.7)
    rng = np.random.default_rng(M)
    x0 = rng.integers(0, 30, size=(6, N)).astype(np.int32)
    netg = api.Network(net)
    g = api.simulate(netg, x0, 1.0, 6, seed=M, stream_id=1, traj_offset=3, max_events=1500, sample_dt=0.001,
                     grid="traj", grad=True, mapping=L.RT_MAP_BLOCK, block_threads=B)
    o = oracle.run(net, x0, 1.0, 6, seed=M, stream_id=1, traj_offset=3, max_events=1500, sample_dt=0.001,
                   want_grid=True, want_grad=True, n_threads=6)
    assert_same(g, o)


def test_block_mapping_finite_horizon_likelihood():
    net = W.random_mass_action(100, 400, seed=77, c_sigma=0.5)
    x0 = W.poisson_x0(100, 8, 78)
    netg = api.Network(net)
    g = api.simulate(netg, x0, 0.01, 9, seed=3, grad=True, mapping=L.RT_MAP_BLOCK, max_events=100000)
    o = oracle.run(net, x0, 0.01, 9, seed=3, want_grad=True, max_events=100000, n_threads=9)
    assert (o["status"] == 0).all()
    assert_same(g, o)


def _overflow_network(M):
    """M - 1 slow first-order conversions among species 1..3 and one fast birth of species 0."""
    rng = np.random.default_rng(M)
    reactions = []
    for _ in range(M - 1):
        a, b = rng.choice([1, 2, 3], size=2, replace=False)
        reactions.append(({int(a): 1}, {int(b): 1}, float(rng.uniform(0.5, 2.0))))
    reactions.append(({}, {0: 1}, 1e6))
    return W._from_lists(4, reactions, "overflow%d" % M)


@pytest.mark.parametrize("grid", [False, True])
@pytest.mark.parametrize("mapping,M", [(L.RT_MAP_WARP, 100), (L.RT_MAP_BLOCK, 700), (L.RT_MAP_BUNDLE, 700)])
def test_overflow_stops_before_the_event(mapping, M, grid):
    """A fast birth drives species 0 to INT32_MAX: the event that would pass it does not fire and
    the run stops with OVERFLOW, with the grid (sampled densely, so the last events cross grid
    points) and the counts as the oracle has them."""
    net = _overflow_network(M)
    x0 = np.array([[2**31 - 60, 50, 50, 50], [2**31 - 7, 10, 10, 10], [5, 50, 50, 50]], np.int32)
    kw = dict(grid="traj", sample_dt=2e-6) if grid else {}
    g = api.simulate(api.Network(net), x0, 1e-3, 3, seed=6, grad=True, mapping=mapping,
                     ctas_per_traj=2 if mapping == L.RT_MAP_BUNDLE else 0, **kw)
    o = oracle.run(net, x0, 1e-3, 3, seed=6, want_grad=True, want_grid=grid, n_threads=3,
                   **({"sample_dt": 2e-6} if grid else {}))
    assert o["status"][:2].tolist() == [oracle.ST_OVERFLOW, oracle.ST_OVERFLOW]
    assert o["status"][2] == oracle.ST_TEND
    assert_same(g, o)
