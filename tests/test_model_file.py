"""The model-file format of the paper's Table 4 (Sec. 5), parsed by the library's host code
through the C ABI (rt_model_parse; no GPU needed)."""
import os

import numpy as np
import pytest

from paper_2103_00405_gb300 import _lib as L
from paper_2103_00405_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))

try:
    L.load()
except ImportError:  # pragma: no cover
    pytest.skip("librandtime not built", allow_module_level=True)

from paper_2103_00405_gb300 import api  # noqa: E402


def _coo(net):
    r = sorted(zip(net.reac_rxn.tolist(), net.reac_sp.tolist(), net.reac_coef.tolist()))
    v = sorted(zip(net.stoi_rxn.tolist(), net.stoi_sp.tolist(), net.stoi_delta.tolist()))
    return r, v


def test_table4_example_is_the_lotka_volterra_model():
    """Table 4's printed example: species A = B = 1000, X -> 2X (10), X + Y -> 2Y (0.01), Y -> 0 (10),
    time = 2, steps = 10000 -- the model the rest of the build calls Lotka-Volterra."""
    m = api.parse_model(open(os.path.join(HERE, "golden", "table4_lotka_volterra.txt")).read())
    ref = W.lotka_volterra(10.0, 0.01, 10.0)
    assert m["names"] == ["A", "B"]
    assert m["x0"].tolist() == [1000, 1000]
    assert m["time"] == 2.0 and m["steps"] == 10000
    assert m["net"].n_species == 2 and m["net"].n_reactions == 3
    assert _coo(m["net"]) == _coo(ref)
    assert np.array_equal(m["net"].c, ref.c)


def test_optional_coefficients_comments_and_species_order():
    text = """
    // comment line
    # init
    B = 5
    # reactions
    A + B -> C : 2.5   // trailing comment
    2 C --> NULL : 0.5
    NULL --> A : 1e-3
    # end
    """
    m = api.parse_model(text)
    assert m["names"] == ["B", "A", "C"] and m["x0"].tolist() == [5, 0, 0]
    assert m["time"] is None and m["steps"] is None
    S = m["net"].dense_reactants()
    V = m["net"].dense_stoich()
    assert S.tolist() == [[1, 1, 0], [0, 0, 2], [0, 0, 0]]
    assert V.tolist() == [[-1, -1, 1], [0, 0, -2], [0, 1, 0]]
    assert m["net"].c.tolist() == [2.5, 0.5, 1e-3]


@pytest.mark.parametrize("text,fragment", [
    ("# reactions\n1 A --> : 1\n", "empty side"),
    ("# reactions\n1 A --> 2 A\n", "expected"),
    ("# reactions\n1 A --> 2 A : -1\n", "rate"),
    ("# init\nA = -3\n# reactions\nA --> NULL : 1\n", "initial count"),
    ("# init\nA = 1\nA = 2\n# reactions\nA --> NULL : 1\n", "twice"),
    ("A --> NULL : 1\n", "outside a section"),
    ("# bogus\n", "unknown section"),
    ("# init\nA = 1\n", "no reactions"),
    ("# reactions\n0 A --> B : 1\n", "coefficient"),
])
def test_malformed_text_is_rejected_with_the_line(text, fragment):
    with pytest.raises(L.RandtimeError) as e:
        api.parse_model(text)
    assert fragment in str(e.value)
