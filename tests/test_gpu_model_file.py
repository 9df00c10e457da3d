"""A model read from Table 4's text format runs on the GPU: the printed example (time = 2,
steps = 10000, output grid time / steps) against the oracle on the same parsed network, bit for
bit, in the three forms of the method."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import _lib as L  # noqa: E402
from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

from test_gpu_parity import assert_same  # noqa: E402

B.build()

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("form,mode", [(L.RT_FORM_INTERNAL, oracle.MODE_EAGER), (L.RT_FORM_ABSOLUTE, oracle.MODE_LAZY),
                                       (L.RT_FORM_RESCALED, oracle.MODE_RESCALED)])
def test_table4_file_simulates_like_the_oracle(form, mode):
    m = api.parse_model(open(os.path.join(HERE, "golden", "table4_lotka_volterra.txt")).read())
    t_end, dt = m["time"], m["time"] / m["steps"]
    n = 8
    g = api.simulate(api.Network(m["net"]), m["x0"], t_end, n, seed=3, sample_dt=dt, grid="traj", grad=True,
                     trace_len=2000, form=form)
    o = oracle.run(m["net"], m["x0"], t_end, n, seed=3, sample_dt=dt, want_grid=True, want_grad=True,
                   trace_len=2000, mode=mode, n_threads=8)
    assert o["grid"].shape[1] == m["steps"] + 1
    assert (o["n_events"] > 100).all()
    assert_same(g, o, keys=("x_final", "n_events", "status", "counts", "grid", "trace_mu", "t_last", "t_internal",
                            "loglik", "trace_t"))
