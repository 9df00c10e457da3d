"""Forbidden channels (Table 2's note: a channel forbidden to fire keeps a frozen internal time),
set with rt_network_set_enabled, against the oracle's enabled mask, bit for bit, in every mapping."""
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

CASES = {
    "small": (W.lotka_volterra(), np.array([1000, 1000], np.int32), 0.3, 20, dict(mapping=L.RT_MAP_THREAD), 0),
    "thread": (W.random_mass_action(6, 12, seed=61), None, 0.5, 30, dict(mapping=L.RT_MAP_THREAD), 0),
    "warp": (W.random_mass_action(16, 64, seed=62, c_sigma=0.5), None, 0.05, 20, dict(mapping=L.RT_MAP_WARP), 0),
    "block": (W.random_mass_action(250, 1000, seed=63), None, 0.02, 4, dict(mapping=L.RT_MAP_BLOCK), 0),
    "bundle": (W.random_mass_action(300, 5000, seed=64), None, 0.002, 3,
               dict(mapping=L.RT_MAP_BUNDLE, ctas_per_traj=3), 0),
    "tree": (W.random_mass_action(300, 5000, seed=65), None, 0.002, 3, dict(form=L.RT_FORM_ABSOLUTE), 1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_forbidden_channels_are_frozen_in_every_mapping(name):
    net, x0, t_end, n, kw, mode = CASES[name]
    if x0 is None:
        x0 = W.poisson_x0(net.n_species, 60, 9)
    en = (np.random.default_rng(len(name)).random(net.n_reactions) > 0.3).astype(np.uint8)
    en[0] = 0
    netg = api.Network(net).set_enabled(en)
    g = api.simulate(netg, x0, t_end, n, seed=4, grad=True, max_events=4000, trace_len=400, **kw)
    o = oracle.run(net, x0, t_end, n, seed=4, want_grad=True, max_events=4000, trace_len=400, enabled=en, mode=mode,
                   n_threads=8)
    assert o["n_events"].min() > 10
    assert_same(g, o)
    assert (g["counts"].cpu().numpy()[:, en == 0] == 0).all()
    # the gradient divides by the network's own rates: forbidden channels get 0
    gc = api.loglik_backward(netg, torch.ones(n, dtype=torch.float64, device="cuda"), g["counts"], g["t_internal"])
    ref = oracle.loglik_backward(np.ones(n), o["counts"], o["t_internal"], net.c)
    assert np.array_equal(gc.cpu().numpy().view(np.int64), ref.view(np.int64))
    assert (gc.cpu().numpy()[en == 0] == 0).all()
    # enabling every channel again restores the unmasked network
    netg.set_enabled(None)
    g2 = api.simulate(netg, x0, t_end, n, seed=4, max_events=4000, **kw)
    o2 = oracle.run(net, x0, t_end, n, seed=4, max_events=4000, mode=mode, n_threads=8)
    assert_same(g2, o2, keys=("x_final", "n_events", "status", "t_last"))


def test_batch_takes_the_setting_of_its_networks():
    items = W.batched_networks(12, m_lo=2, m_hi=300, seed=81, t_lo=0.05, t_hi=0.2)
    ens = [(np.arange(it.net.n_reactions) % 3 != 1).astype(np.uint8) for it in items]
    batch = api.Batch([it.net for it in items], enabled=ens)
    x0 = torch.from_numpy(np.concatenate([it.x0 for it in items])).cuda()
    t_end = torch.tensor([it.t_end for it in items], dtype=torch.float64).cuda()
    out = batch.run(x0, t_end, 2, seed=5, max_events=3000, outputs=batch.outputs(2, grad=True))
    torch.cuda.synchronize()
    for i, (it, e) in enumerate(zip(items, ens)):
        o = oracle.run(it.net, it.x0, it.t_end, 2, seed=5, stream_id=i, max_events=3000, want_grad=True, enabled=e)
        assert np.array_equal(batch.x_final_of(out, i, 2).cpu().numpy(), o["x_final"])
        assert np.array_equal(batch.per_channel_of(out, "counts", i, 2).cpu().numpy(), o["counts"])
