"""GPU path against the CPU oracle, element by element, through the C ABI.

The bar: integers (states, counts, event numbers, statuses, grids) identical;
binary64 outputs (times, internal times, log-likelihoods) identical bit for bit,
because both sides perform the same IEEE operations in the same order.  The
stated tolerance for times is 1e-12 relative; every comparison below uses 0.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_00405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts skip the GPU suite
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import _lib as L  # noqa: E402
from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

B.build()

KEYS_INT = ("x_final", "n_events", "status", "counts", "grid")
KEYS_F64 = ("t_last", "t_internal", "loglik")


def assert_same(gpu: dict, ora: dict, keys=KEYS_INT + KEYS_F64, idx=None):
    torch.cuda.synchronize()
    for k in keys:
        if k not in ora or k not in gpu:
            continue
        g = gpu[k].cpu().numpy()
        o = ora[k]
        if idx is not None:
            g = g[idx]
        if g.dtype == np.float64:
            same = (g.view(np.int64) == o.view(np.int64)) | (np.isnan(g) & np.isnan(o))
            assert same.all(), (k, np.argwhere(~same)[:5], g[~same][:5], o[~same][:5])
        else:
            assert np.array_equal(g, o.astype(g.dtype)), (k, np.argwhere(g != o)[:5])


def run_both(net, x0, t_end, n_traj, grad=False, grid=False, nthreads=16, **kw):
    netg = api.Network(net)
    g = api.simulate(netg, x0, t_end, n_traj, grid="traj" if grid else "none", grad=grad, **kw)
    okw = {k: v for k, v in kw.items() if k in ("seed", "stream_id", "traj_offset", "max_events", "sample_dt")}
    o = oracle.run(net, x0, t_end, n_traj, want_grid=grid, want_grad=grad, n_threads=nthreads, **okw)
    return g, o


# ---------------------------------------------------------------------------------
# Random draws and logarithm
# ---------------------------------------------------------------------------------

def test_philox_device_equals_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
    out = api.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), int(key[0]), int(key[1])).cpu().numpy()
    out = out.view(np.uint32).reshape(-1, 4)
    lib = oracle.load()
    for i in range(0, 5000, 7):
        assert out[i].tolist() == oracle.philox4x32_10(ctr[i], key, lib).tolist()


def test_log_device_equals_oracle_bitwise():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(0, 1, 40000), np.exp(rng.uniform(-745, 709, 40000)),
                        1 + rng.uniform(-1e-6, 1e-6, 5000), (2 * rng.integers(0, 2**52, 20000) + 1) * 2.0**-53,
                        [5e-324, 2.2250738585072014e-308, 1.0, 2.0, 0.5, 1 - 2**-53, 1 + 2**-52,
                         1.7976931348623157e308, math.sqrt(2), 2**-1022]])
    y = api.log_eval(torch.from_numpy(x).cuda()).cpu().numpy()
    lib = oracle.load()
    ref = np.array([lib.oracle_rt_log(float(v)) for v in x])
    bad = np.flatnonzero(y.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, (x[bad[:5]], y[bad[:5]], ref[bad[:5]])


def test_log_device_within_one_ulp_of_cuda_log():
    rng = np.random.default_rng(3)
    x = torch.from_numpy(np.exp(rng.uniform(-700, 700, 100000))).cuda()
    y = api.log_eval(x)
    ref = torch.log(x)
    ulp = torch.from_numpy(np.spacing(np.abs(ref.cpu().numpy()))).cuda()
    assert ((y - ref).abs() <= ulp).all()


def test_exp1_draws_equal_oracle_bitwise():
    rng = np.random.default_rng(4)
    n = 20000
    traj = rng.integers(0, 2**40, n, dtype=np.uint64)
    ch = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    idx = rng.integers(0, 2**31, n, dtype=np.uint64)
    seed, stream = 0xDEADBEEF12345, 7
    u, e = api.draw_exp1(seed, traj, ch, idx, stream)
    u, e = u.cpu().numpy(), e.cpu().numpy()
    lib = oracle.load()
    for i in range(0, n, 3):
        args = (seed, int(traj[i]), int(ch[i]), int(idx[i]), stream)
        assert u[i] == lib.oracle_uniform(*args)
        assert e[i] == lib.oracle_exp1(*args)


# ---------------------------------------------------------------------------------
# Whole trajectories, thread-per-trajectory mapping
# ---------------------------------------------------------------------------------

def test_lotka_volterra_64_trajectories_bit_exact():
    """Lotka-Volterra of Table 4, c = (10, 0.01, 10), X0 = (1000, 1000), t_end = 5, grid 0.01, seed 1."""
    cfg = W.lv_config(64)
    g, o = run_both(cfg["net"], cfg["x0"], cfg["t_end"], 64, grad=True, grid=True, seed=1, sample_dt=0.01)
    assert g["grid"].shape == (64, 501, 2)
    assert_same(g, o)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_ensemble_networks_bit_exact_ragged(which):
    """Lotka-Volterra, birth-death and dimerisation to t_end = 10, a ragged trajectory count."""
    c = W.ensemble_configs(300)[which]
    g, o = run_both(c["net"], c["x0"], c["t_end"], 300, grad=True, grid=True, seed=c["seed"], sample_dt=0.05,
                    max_events=c["max_events"])
    assert_same(g, o)


@pytest.mark.parametrize("seed", range(6))
def test_random_small_networks_bit_exact(seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(1, 17))
    N = int(rng.integers(1, 7))
    net = W.random_mass_action(N, M, seed=1000 + seed, c_sigma=0.8)
    x0 = rng.integers(0, 40, size=(97, N)).astype(np.int32)
    g, o = run_both(net, x0, 3.0, 97, grad=True, grid=True, seed=seed + 17, stream_id=seed, traj_offset=1000 * seed,
                    max_events=20000, sample_dt=0.1)
    assert_same(g, o)


@pytest.mark.parametrize("M,N", [(m, n) for m in range(1, 5) for n in range(1, 6)])
def test_small_networks_every_shape_bit_exact(M, N):
    """Every M <= 4 with N <= 4 runs the register kernel (network as a kernel parameter, X in
    registers); N = 5 the shared-memory thread kernel.  Per-trajectory X0, grids and gradients."""
    net = W.random_mass_action(N, M, seed=7000 + 10 * M + N, c_sigma=0.8)
    rng = np.random.default_rng(M * 10 + N)
    x0 = rng.integers(0, 60, size=(161, N)).astype(np.int32)
    g, o = run_both(net, x0, 2.0, 161, grad=True, grid=True, seed=M + N, stream_id=3, traj_offset=55,
                    max_events=20000, sample_dt=0.1)
    assert_same(g, o)


@pytest.mark.parametrize("B", [32, 64, 128])
def test_block_size_does_not_change_results(B):
    cfg = W.lv_config(100)
    netg = api.Network(cfg["net"])
    g = api.simulate(netg, cfg["x0"], 1.0, 100, seed=3, grad=True, mapping=L.RT_MAP_THREAD, block_threads=B)
    o = oracle.run(cfg["net"], cfg["x0"], 1.0, 100, seed=3, want_grad=True, n_threads=16)
    assert_same(g, o)


def test_moments_equal_sums_of_oracle_grids():
    c = W.ensemble_configs(500)[2]
    netg = api.Network(c["net"])
    g = api.simulate(netg, c["x0"], 10.0, 500, seed=1, sample_dt=0.1, grid="moments", max_events=c["max_events"])
    o = oracle.run(c["net"], c["x0"], 10.0, 500, seed=1, sample_dt=0.1, want_grid=True, n_threads=16)
    grid = o["grid"].astype(np.int64)
    assert np.array_equal(g["grid_sum"].cpu().numpy(), grid.sum(0))
    assert np.array_equal(g["grid_sumsq"].cpu().numpy(), (grid ** 2).sum(0))
    assert np.array_equal(g["grid_count"].cpu().numpy(), np.full(grid.shape[1], 500))


@pytest.mark.parametrize("sample_dt", [0.02, 0.01, 0.001])
def test_cluster_shared_moments_equal_sums_of_oracle_grids(sample_dt):
    """Grids of 501, 1001 and 10001 points: the moment table is split across clusters of 2, 4 and
    8 blocks; 300 trajectories leave the last cluster partly without trajectories."""
    c = W.ensemble_configs(300)[2]
    netg = api.Network(c["net"])
    g = api.simulate(netg, c["x0"], 10.0, 300, seed=7, sample_dt=sample_dt, grid="moments",
                     max_events=c["max_events"])
    o = oracle.run(c["net"], c["x0"], 10.0, 300, seed=7, sample_dt=sample_dt, want_grid=True, n_threads=16)
    grid = o["grid"].astype(np.int64)
    assert np.array_equal(g["grid_sum"].cpu().numpy(), grid.sum(0))
    assert np.array_equal(g["grid_sumsq"].cpu().numpy(), (grid ** 2).sum(0))
    assert np.array_equal(g["grid_count"].cpu().numpy(), np.full(grid.shape[1], 300))


def test_edge_cases_bit_exact():
    lv = W.lotka_volterra()
    # no trajectories
    g = api.simulate(api.Network(lv), [1000, 1000], 1.0, 0)
    assert g["x_final"].shape == (0, 2)
    # zero event budget, zero horizon, infinite horizon with a cap
    for kw in (dict(t_end=5.0, max_events=0), dict(t_end=0.0), dict(t_end=math.inf, max_events=777)):
        t_end = kw.pop("t_end")
        g, o = run_both(lv, np.array([1000, 1000], np.int32), t_end, 33, grad=True, seed=5, **kw)
        assert_same(g, o)
    # absorption (pure death), overflow (fast birth near INT32_MAX), negative initial counts
    death = W._from_lists(1, [({0: 1}, {}, 1.0)], "death")
    g, o = run_both(death, [7], 100.0, 40, grad=True, seed=2)
    assert (o["status"] == oracle.ST_ABSORBED).all()
    assert_same(g, o)
    birth = W.pure_birth(1e6)
    g, o = run_both(birth, [2**31 - 5], math.inf, 40, seed=2)
    assert (o["status"] == oracle.ST_OVERFLOW).all()
    assert_same(g, o)
    x0 = np.array([[5], [-1], [0]], np.int32)
    g, o = run_both(W.birth_death(), x0, 1.0, 3, grad=True, grid=True, seed=2, sample_dt=0.5)
    assert o["status"][1] == oracle.ST_BAD_X0
    assert_same(g, o)


def test_full_size_ensemble_sampled_against_oracle():
    """2^20 trajectories of each ensemble network to t_end = 10 (the benchmarked launch), with
    16 trajectories spread over the range re-run one by one in the oracle."""
    n = 1 << 20
    for c in W.ensemble_configs(n):
        netg = api.Network(c["net"])
        g = api.simulate(netg, c["x0"], c["t_end"], n, seed=c["seed"], sample_dt=0.01, grid="moments",
                         max_events=c["max_events"])
        torch.cuda.synchronize()
        status = g["status"].cpu().numpy()
        xf = g["x_final"].cpu().numpy().astype(np.int64)
        # the last grid point is t_end: its sum is the sum of final states of trajectories that reached t_end
        known = (status == 0) | (status == 2)
        assert np.array_equal(g["grid_sum"][-1].cpu().numpy(), xf[known].sum(0))
        assert g["grid_count"][-1].item() == known.sum()
        assert np.array_equal(g["grid_sum"][0].cpu().numpy(), n * c["x0"].astype(np.int64))
        odd = np.flatnonzero(status != 0)[:4]  # capped, absorbed or overflowed trajectories, if any
        for j in list(np.linspace(0, n - 1, 16).astype(np.int64)) + list(odd):
            o = oracle.run(c["net"], c["x0"], c["t_end"], 1, seed=c["seed"], traj_offset=int(j),
                           max_events=c["max_events"])
            for k in ("x_final", "n_events", "status", "t_last"):
                gv = g[k][j].cpu().numpy()
                ov = o[k][0]
                if gv.dtype == np.float64:
                    assert gv.view(np.int64) == ov.view(np.int64), (c["net"].name, j, k)
                else:
                    assert np.array_equal(gv, ov), (c["net"].name, j, k, gv, ov)


def test_backward_kernel_and_autograd_against_oracle():
    cfg = W.grad_config(512)
    net, x0 = cfg["net"], cfg["x0"]
    c = torch.tensor(net.c, dtype=torch.float64, requires_grad=True)
    ll = api.LogLik.apply(c, net, x0, 1.0, 512, 1, 0, 200000)
    w = torch.linspace(-1, 1, 512, dtype=torch.float64, device=ll.device)
    (ll * w).sum().backward()
    o = oracle.run(net, x0, 1.0, 512, seed=1, max_events=200000, want_grad=True, n_threads=16)
    assert np.array_equal(ll.detach().cpu().numpy().view(np.int64), o["loglik"].view(np.int64))
    ref = oracle.loglik_backward(w.cpu().numpy(), o["counts"], o["t_internal"], net.c)
    np.testing.assert_allclose(c.grad.numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # closed form, independent of either reduction order
    closed = ((o["counts"] - o["t_internal"]) / net.c * w.cpu().numpy()[:, None]).sum(0)
    np.testing.assert_allclose(c.grad.numpy(), closed, rtol=1e-9, atol=1e-9 * np.abs(closed).max())
