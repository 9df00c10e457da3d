"""Time-dependent rates c_k(t) = c_k (1 + beta_k t) (Sec. 6, Eq. 29; rt_network_set_rate_slopes)
on the thread mapping (M <= 16) and the warp mapping (M <= 256) against the oracle, bit for bit,
through the C ABI."""
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


@pytest.mark.parametrize("M,N", [(2, 1), (3, 2), (6, 4), (12, 6), (16, 5)])
def test_ramped_rates_bit_exact(M, N):
    net = W.birth_death(40.0, 1.0) if M == 2 else W.lotka_volterra(1.0, 0.05, 1.0) if M == 3 else \
        W.random_mass_action(N, M, seed=900 + M, c_sigma=0.6)
    rng = np.random.default_rng(M)
    beta = np.where(rng.random(M) < 0.3, 0.0, rng.uniform(0.1, 3.0, M))
    x0 = np.array([0], np.int32) if M == 2 else np.array([20, 20], np.int32) if M == 3 else W.poisson_x0(N, 25, M)
    n = 300
    netg = api.Network(net).set_rate_slopes(beta)
    g = api.simulate(netg, x0, 1.5, n, seed=M, stream_id=2, traj_offset=3, max_events=100000, grad=True,
                     grid="traj", sample_dt=0.1, trace_len=400)
    o = oracle.run(net, x0, 1.5, n, seed=M, stream_id=2, traj_offset=3, max_events=100000, want_grad=True,
                   want_grid=True, sample_dt=0.1, trace_len=400, beta=beta, n_threads=16)
    assert o["n_events"].mean() > 10
    assert_same(g, o)
    assert_trace(g, o)


@pytest.mark.parametrize("M,N", [(17, 6), (40, 10), (64, 16), (100, 30), (256, 64)])
def test_ramped_rates_on_the_warp_mapping_bit_exact(M, N):
    """Networks above 16 reactions run a warp per trajectory by default (trace, grid, counts,
    internal times, likelihood); then moments under an event cap on the explicitly requested warp
    mapping."""
    net = W.random_mass_action(N, M, seed=950 + M, c_sigma=0.6)
    rng = np.random.default_rng(M)
    beta = np.where(rng.random(M) < 0.3, 0.0, rng.uniform(0.1, 3.0, M))
    x0 = W.poisson_x0(N, 25, M)
    n = 67  # a ragged last block of warps
    netg = api.Network(net).set_rate_slopes(beta)
    t_end = 0.6 if M <= 64 else 0.25
    g = api.simulate(netg, x0, t_end, n, seed=M, stream_id=1, traj_offset=5, max_events=100000, grad=True,
                     grid="traj", sample_dt=0.05, trace_len=300)
    o = oracle.run(net, x0, t_end, n, seed=M, stream_id=1, traj_offset=5, max_events=100000, want_grad=True,
                   want_grid=True, sample_dt=0.05, trace_len=300, beta=beta, n_threads=16)
    assert o["n_events"].mean() > 10
    assert_same(g, o)
    assert_trace(g, o)
    # moments, event cap and an explicit warp mapping
    m = api.simulate(netg, x0, t_end, n, seed=M, max_events=40, sample_dt=0.05, grid="moments",
                     mapping=L.RT_MAP_WARP, lanes_per_traj=32)
    om = oracle.run(net, x0, t_end, n, seed=M, max_events=40, sample_dt=0.05, want_grid=True, beta=beta,
                    n_threads=16)
    grid = om["grid"].astype(np.int64)
    known = grid >= 0
    assert np.array_equal(m["grid_sum"].cpu().numpy(), np.where(known, grid, 0).sum(0))
    assert np.array_equal(m["grid_count"].cpu().numpy(), known[:, :, 0].sum(0))
    assert np.array_equal(m["n_events"].cpu().numpy(), om["n_events"])


def test_zero_slopes_give_the_constant_rate_path_and_moments():
    net = W.random_mass_action(5, 9, seed=95)
    x0 = W.poisson_x0(5, 20, 96)
    netg = api.Network(net)
    a = api.simulate(netg, x0, 1.0, 500, seed=3, grad=True, mapping=L.RT_MAP_THREAD)
    netg.set_rate_slopes(np.zeros(9))
    b = api.simulate(netg, x0, 1.0, 500, seed=3, grad=True, mapping=L.RT_MAP_THREAD)
    torch.cuda.synchronize()
    for k in ("x_final", "n_events", "counts"):
        assert torch.equal(a[k], b[k]), k
    for k in ("t_last", "t_internal", "loglik"):
        assert torch.equal(a[k].view(torch.int64), b[k].view(torch.int64)), k
    # moments of a ramped birth against the oracle's grid
    birth = W.pure_birth(10.0)
    gb = api.Network(birth).set_rate_slopes([0.5])
    m = api.simulate(gb, [0], 3.0, 4000, seed=1, sample_dt=0.5, grid="moments")
    o = oracle.run(birth, [0], 3.0, 4000, seed=1, sample_dt=0.5, want_grid=True, beta=[0.5], n_threads=16)
    grid = o["grid"].astype(np.int64)
    assert np.array_equal(m["grid_sum"].cpu().numpy(), grid.sum(0))
    assert np.array_equal(m["grid_sumsq"].cpu().numpy(), (grid ** 2).sum(0))


def test_time_dependent_rates_are_refused_where_unsupported():
    netg = api.Network(W.random_mass_action(10, 40, seed=97)).set_rate_slopes(np.full(40, 0.5))
    x0 = W.poisson_x0(10, 20, 1)
    for kw in (dict(mapping=L.RT_MAP_THREAD), dict(mapping=L.RT_MAP_BLOCK), dict(form=L.RT_FORM_ABSOLUTE),
               dict(form=L.RT_FORM_RESCALED), dict(mapping=L.RT_MAP_WARP, lanes_per_traj=8)):
        with pytest.raises(L.RandtimeError):
            api.simulate(netg, x0, 1.0, 2, **kw)
    big = api.Network(W.random_mass_action(60, 300, seed=98)).set_rate_slopes(np.full(300, 0.5))
    with pytest.raises(L.RandtimeError):
        api.simulate(big, W.poisson_x0(60, 20, 1), 1.0, 2)
    with pytest.raises(L.RandtimeError):
        api.Network(W.birth_death()).set_rate_slopes([-1.0, 0.0])
