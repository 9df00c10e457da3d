"""Event by event: the GPU's per-event trace (fired channel, event time) against the oracle's, bit
for bit, in every mapping -- the small-network, thread, warp, block and bundle kernels and the
batched kernel -- through the C ABI.  The trace is the event sequence of Table 2's loop: which
channel j fired at each step and the time t after the update t += dt."""
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

B.build()


def assert_trace(g, o, idx=None):
    torch.cuda.synchronize()
    mu, tt = g["trace_mu"].cpu().numpy(), g["trace_t"].cpu().numpy()
    if idx is not None:
        mu, tt = mu[idx], tt[idx]
    bad = np.argwhere(mu != o["trace_mu"])
    assert bad.size == 0, ("first differing (trajectory, event)", bad[:3], mu[tuple(bad[0])], o["trace_mu"][tuple(bad[0])])
    badt = np.argwhere(tt.view(np.int64) != o["trace_t"].view(np.int64))
    assert badt.size == 0, ("event times differ", badt[:3])


CASES = {
    # name: (network, x0, t_end, n_traj, mapping, extra simulate kwargs)
    "small": (W.lotka_volterra(), np.array([1000, 1000], np.int32), 0.2, 24, L.RT_MAP_THREAD, {}),
    "thread": (W.random_mass_action(6, 12, seed=31), None, 0.5, 40, L.RT_MAP_THREAD, {}),
    "warp": (W.random_mass_action(16, 64, seed=32, c_sigma=0.5), None, 0.02, 20, L.RT_MAP_WARP, {}),
    "block": (W.random_mass_action(250, 1000, seed=33), None, 0.02, 6, L.RT_MAP_BLOCK, {}),
    "bundle": (W.random_mass_action(300, 5000, seed=34), None, 0.002, 3, L.RT_MAP_BUNDLE, dict(ctas_per_traj=3)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("grad", [False, True])
def test_trace_equals_oracle_in_every_mapping(name, grad):
    net, x0, t_end, n, mapping, kw = CASES[name]
    if x0 is None:
        x0 = W.poisson_x0(net.n_species, 60, 7)
    K = 1500
    netg = api.Network(net)
    g = api.simulate(netg, x0, t_end, n, seed=5, stream_id=2, traj_offset=11, max_events=3000, grad=grad,
                     mapping=mapping, trace_len=K, **kw)
    o = oracle.run(net, x0, t_end, n, seed=5, stream_id=2, traj_offset=11, max_events=3000, want_grad=grad,
                   trace_len=K, n_threads=16)
    assert o["n_events"].min() > 20, "too few events to exercise the trace"
    assert_trace(g, o)
    assert_same(g, o)


def test_trace_tail_and_short_trace():
    """A trace shorter than the run holds the first trace_len events; a longer one ends in -1 / 0."""
    net, x0 = W.birth_death(), np.array([0], np.int32)
    netg = api.Network(net)
    for K in (7, 5000):
        g = api.simulate(netg, x0, 2.0, 33, seed=3, trace_len=K)
        o = oracle.run(net, x0, 2.0, 33, seed=3, trace_len=K, n_threads=4)
        assert_trace(g, o)
        if K == 5000:
            ev = o["n_events"]
            assert (ev < K).all() and all((o["trace_mu"][j, ev[j]:] == -1).all() for j in range(33))


def test_batched_trace_and_likelihood_per_network():
    """One persistent launch over uneven networks with the trace and the log-likelihood outputs:
    every network's trajectories equal the oracle's (stream id = global index)."""
    items = W.batched_networks(40, m_lo=1, m_hi=600, seed=91, t_lo=0.02, t_hi=0.1)
    sid = np.arange(100, 140, dtype=np.uint32)
    batch = api.Batch([it.net for it in items], stream_ids=sid)
    x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).cuda()
    t_end = torch.tensor([it.t_end for it in items], dtype=torch.float64).cuda()
    n, K = 2, 400
    out = batch.run(x0, t_end, n, seed=8, max_events=2500, outputs=batch.outputs(n, grad=True, trace_len=K))
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        o = oracle.run(it.net, it.x0, it.t_end, n, seed=8, stream_id=int(sid[i]), max_events=2500,
                       want_grad=True, trace_len=K, n_threads=2)
        g = dict(x_final=batch.x_final_of(out, i, n), n_events=out["n_events"][i], status=out["status"][i],
                 t_last=out["t_last"][i], loglik=out["loglik"][i],
                 counts=batch.per_channel_of(out, "counts", i, n),
                 t_internal=batch.per_channel_of(out, "t_internal", i, n),
                 trace_mu=out["trace_mu"][i], trace_t=out["trace_t"][i])
        assert_same(g, o)
        assert_trace(g, o)


@pytest.mark.slow
def test_large_network_full_size_trajectory_event_by_event():
    """The N = 1e4, M = 1e6 network at its benchmarked launch (bundle mapping, library-chosen block
    count): one trajectory's first 3000 events against the oracle, event by event, with the
    counts, internal times and final state (the paths the scan takes only later in a run -- the
    refreshed sum of propensities every 64 events, the threshold and the exact re-scan -- all
    occur within these events)."""
    cfg = W.large_network_config(max_events=3000)
    net, x0 = cfg["net"], cfg["x0"]
    netg = api.Network(net)
    g = api.simulate(netg, x0, math.inf, 1, seed=1, traj_offset=5, max_events=3000, grad=True,
                     mapping=L.RT_MAP_BUNDLE, trace_len=3000)
    o = oracle.run(net, x0, math.inf, 1, seed=1, traj_offset=5, max_events=3000, want_grad=True, trace_len=3000,
                   n_threads=1)
    assert o["n_events"][0] == 3000
    assert_trace(g, o)
    assert_same(g, o, keys=("x_final", "n_events", "status", "counts", "t_last", "t_internal"))


def test_batch_shared_memory_limit_survives_a_smaller_batch():
    """The persistent kernel's dynamic shared-memory limit is shared by every batch: creating a
    smaller batch (still above the 48 KB default) after a larger one must not break the larger
    one's launches or graph replays."""
    def items(n_species, seed):  # block-class networks whose species table alone is > 48 KB
        net = W.random_mass_action(n_species, 3000, seed=seed)
        return [W.BatchItem(net, W.poisson_x0(n_species, 50, seed + 1), 0.003)]

    big, small = items(15000, 5), items(13000, 6)

    def mk(items):
        b = api.Batch([it.net for it in items], block_threads=512)
        x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).cuda()
        te = torch.tensor([it.t_end for it in items], dtype=torch.float64).cuda()
        return b, x0, te

    bb, bx, bt = mk(big)
    graph, gout = bb.capture(bx, bt, 1, seed=2, max_events=200)
    sb, sx, st = mk(small)
    sb.run(sx, st, 1, seed=2, max_events=200)
    out = bb.run(bx, bt, 1, seed=2, max_events=200)  # the larger batch after the smaller one was made
    graph.replay()
    torch.cuda.synchronize()
    for i, it in enumerate(big):
        o = oracle.run(it.net, it.x0, it.t_end, 1, seed=2, stream_id=i, max_events=200, n_threads=1)
        assert np.array_equal(bb.x_final_of(out, i, 1).cpu().numpy(), o["x_final"])
        assert np.array_equal(bb.x_final_of(gout, i, 1).cpu().numpy(), o["x_final"])


def test_fp64_probe_measures_a_plausible_rate():
    r = api.fp64_probe(iters=256, repeats=1)
    assert 1e10 < r < 5e12, r
