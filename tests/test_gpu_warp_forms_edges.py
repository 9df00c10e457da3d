"""Edge cases of the warp kernels of Table 3's form and of time-dependent rates (networks of
17 to 256 reactions): absorption, the int32 range check, negative initial counts, a zero
horizon and a zero event budget, against the oracle bit for bit."""
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

M = 20
# 20 first-order decays A_i -> 0: every trajectory is absorbed
DEATH = W._from_lists(M, [({i: 1}, {}, 0.5 + 0.1 * i) for i in range(M)], "death20")
# 20 births 0 -> A_i close to the int32 limit: the range check stops every trajectory
BIRTH = W._from_lists(M, [({}, {i: 1}, 1e6) for i in range(M)], "birth20")
BETA = np.linspace(0.0, 2.0, M)


def _cases():
    yield "rescaled", dict(form=L.RT_FORM_RESCALED), dict(mode=oracle.MODE_RESCALED), None
    yield "tdep", dict(), dict(beta=BETA), BETA


@pytest.mark.parametrize("name,gkw,okw,beta", list(_cases()))
def test_warp_form_edges(name, gkw, okw, beta):
    def net_of(spec):
        n = api.Network(spec)
        return n.set_rate_slopes(beta) if beta is not None else n

    # absorption, with counts, internal times and the likelihood to a finite horizon
    x0 = np.arange(1, M + 1, dtype=np.int32)
    g = api.simulate(net_of(DEATH), x0, 50.0, 37, seed=3, grad=True, grid="traj", sample_dt=5.0, **gkw)
    o = oracle.run(DEATH, x0, 50.0, 37, seed=3, want_grad=True, want_grid=True, sample_dt=5.0, n_threads=8, **okw)
    assert (o["status"] == oracle.ST_ABSORBED).all()
    assert_same(g, o)
    # the int32 range check
    xb = np.full(M, 2**31 - 4, np.int32)
    g = api.simulate(net_of(BIRTH), xb, math.inf, 9, seed=2, max_events=1000, **gkw)
    o = oracle.run(BIRTH, xb, math.inf, 9, seed=2, max_events=1000, n_threads=8, **okw)
    assert (o["status"] == oracle.ST_OVERFLOW).all()
    assert_same(g, o, keys=("x_final", "n_events", "status", "t_last"))
    # a negative initial count in one trajectory (per-trajectory X0), a zero horizon, no events
    xp = np.tile(x0, (3, 1))
    xp[1, 7] = -1
    g = api.simulate(net_of(DEATH), xp, 10.0, 3, seed=4, grad=True, **gkw)
    o = oracle.run(DEATH, xp, 10.0, 3, seed=4, want_grad=True, n_threads=8, **okw)
    assert o["status"][1] == oracle.ST_BAD_X0
    assert_same(g, o)
    for t_end, cap in ((0.0, 100), (10.0, 0)):
        g = api.simulate(net_of(DEATH), x0, t_end, 5, seed=6, max_events=cap, grad=True, **gkw)
        o = oracle.run(DEATH, x0, t_end, 5, seed=6, max_events=cap, want_grad=True, n_threads=8, **okw)
        assert_same(g, o)
