"""Batched mode (one persistent launch over many networks of uneven size) against the CPU
oracle, network by network, bit for bit; CUDA-graph capture and replay."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_00405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

B.build()


def make_batch(n_nets, m_hi, seed, **policy):
    items = W.batched_networks(n_nets, m_lo=1, m_hi=m_hi, seed=seed, t_lo=0.05, t_hi=0.3)
    batch = api.Batch([it.net for it in items], **policy)
    x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).cuda()
    t_end = torch.tensor([it.t_end for it in items], dtype=torch.float64).cuda()
    return items, batch, x0, t_end


def check_against_oracle(items, batch, out, n_traj, max_events, seed):
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        o = oracle.run(it.net, it.x0, it.t_end, n_traj, seed=seed, stream_id=i, max_events=max_events, n_threads=4)
        assert np.array_equal(batch.x_final_of(out, i, n_traj).cpu().numpy(), o["x_final"]), i
        assert np.array_equal(out["n_events"][i].cpu().numpy(), o["n_events"]), i
        assert np.array_equal(out["status"][i].cpu().numpy(), o["status"]), i
        assert np.array_equal(out["t_last"][i].cpu().numpy().view(np.int64), o["t_last"].view(np.int64)), i


@pytest.mark.parametrize("policy", [dict(), dict(thread_max_m=4, warp_max_m=64, block_threads=256),
                                    dict(thread_max_m=0, warp_max_m=0),
                                    dict(warp_max_m=64, block_threads=128)])  # up to 16 channels per thread
def test_batch_bit_exact_per_network(policy):
    items, batch, x0, t_end = make_batch(60, 1200, seed=5, **policy)
    info = batch.info()
    assert info["n_thread"] + info["n_warp"] + info["n_block"] == 60
    out = batch.run(x0, t_end, 3, seed=7, max_events=3000)
    check_against_oracle(items, batch, out, 3, 3000, 7)


def test_batch_equals_per_network_launches():
    items, batch, x0, t_end = make_batch(24, 300, seed=9)
    out = batch.run(x0, t_end, 4, seed=2, max_events=2000)
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        g = api.simulate(api.Network(it.net), it.x0, it.t_end, 4, seed=2, stream_id=i, max_events=2000)
        torch.cuda.synchronize()
        assert torch.equal(batch.x_final_of(out, i, 4), g["x_final"])
        assert torch.equal(out["n_events"][i], g["n_events"])


def test_batch_graph_capture_replays_identically():
    items, batch, x0, t_end = make_batch(30, 800, seed=11)
    graph, out = batch.capture(x0, t_end, 2, seed=4, max_events=2500)
    graph.replay()
    torch.cuda.synchronize()
    first = {k: v.clone() for k, v in out.items()}
    graph.replay()
    torch.cuda.synchronize()
    for k in out:
        assert torch.equal(out[k], first[k])
    check_against_oracle(items, batch, out, 2, 2500, 4)


def test_full_size_batch_sampled_against_oracle():
    """The benchmarked batch: 4096 networks, M ~ U{4..4096}, one trajectory each, 20000-event cap,
    in one graph-captured launch; 12 networks spread over the batch (the largest included) are
    re-run one by one in the oracle."""
    items = W.batched_networks(4096)
    batch = api.Batch([it.net for it in items])
    x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).cuda()
    t_end = torch.tensor([it.t_end for it in items], dtype=torch.float64).cuda()
    graph, out = batch.capture(x0, t_end, 1, seed=1, max_events=20000)
    graph.replay()
    torch.cuda.synchronize()
    ms = np.array([it.net.n_reactions for it in items])
    picks = sorted(set(np.linspace(0, 4095, 11).astype(int).tolist() + [int(ms.argmax())]))
    for i in picks:
        it = items[i]
        o = oracle.run(it.net, it.x0, it.t_end, 1, seed=1, stream_id=i, max_events=20000, n_threads=1)
        assert np.array_equal(batch.x_final_of(out, i, 1).cpu().numpy(), o["x_final"]), i
        assert np.array_equal(out["n_events"][i].cpu().numpy(), o["n_events"]), i
        assert np.array_equal(out["status"][i].cpu().numpy(), o["status"]), i
        assert np.array_equal(out["t_last"][i].cpu().numpy().view(np.int64), o["t_last"].view(np.int64)), i
