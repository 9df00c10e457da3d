"""Host-side checks that need no GPU: the C ABI library loads and exports every
symbol include/randtime.h declares, argument validation returns the documented
codes before any device work, and the seeded input generators are deterministic."""
import ctypes
import os

import numpy as np
import pytest

from paper_2103_00405_gb300 import build as B
from paper_2103_00405_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "randtime.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2103_00405_gb300 import _lib
    _lib.load()
    return _lib


def test_library_exports_every_declared_symbol(L):
    lib = L.load()
    declared = L.declared_symbols(HEADER)
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    bound = {name for name, _, _ in L.SIGNATURES}
    assert set(declared) == bound


def test_grid_len_rule(L):
    lib = L.load()
    assert lib.rt_grid_len(5.0, 0.01) == 501
    assert lib.rt_grid_len(10.0, 0.01) == 1001
    assert lib.rt_grid_len(0.0, 0.1) == 1
    assert lib.rt_grid_len(1.0, 0.0) == 0
    assert lib.rt_grid_len(float("inf"), 0.1) == 0


def _create(L, N, M, reac, stoi, c):
    lib = L.load()
    reac = np.array(reac, np.int32).reshape(-1, 3)
    stoi = np.array(stoi, np.int32).reshape(-1, 3)
    c = np.asarray(c, np.float64)
    arrs = [np.ascontiguousarray(reac[:, i]) for i in range(3)] + [np.ascontiguousarray(stoi[:, i]) for i in range(3)]
    p = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
    h = ctypes.c_void_p()
    rc = lib.rt_network_create(N, M, len(reac), p[0], p[1], p[2], len(stoi), p[3], p[4], p[5],
                               c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
    return rc, lib.rt_last_error().decode()


@pytest.mark.parametrize("case,code", [
    (dict(N=0, M=1, reac=[], stoi=[], c=[1.0]), -1),
    (dict(N=1, M=0, reac=[], stoi=[], c=[]), -1),
    (dict(N=1, M=1, reac=[[0, 1, 1]], stoi=[], c=[1.0]), -1),            # species out of range
    (dict(N=1, M=1, reac=[[1, 0, 1]], stoi=[], c=[1.0]), -1),            # reaction out of range
    (dict(N=1, M=1, reac=[[0, 0, 0]], stoi=[], c=[1.0]), -1),            # zero coefficient
    (dict(N=1, M=1, reac=[[0, 0, 3]], stoi=[], c=[1.0]), -2),            # order 3
    (dict(N=3, M=1, reac=[[0, 0, 1], [0, 1, 1], [0, 2, 1]], stoi=[], c=[1.0]), -2),  # A+B+C
    (dict(N=1, M=1, reac=[[0, 0, 1], [0, 0, 2]], stoi=[], c=[1.0]), -2),  # duplicates summing to 3
    (dict(N=1, M=1, reac=[], stoi=[], c=[-1.0]), -1),                   # negative rate
    (dict(N=1, M=1, reac=[], stoi=[], c=[float("nan")]), -1),           # NaN rate
    (dict(N=1, M=1, reac=[], stoi=[], c=[float("inf")]), -1),
    (dict(N=2, M=1, reac=[[0, 0, 1]], stoi=[[0, 1, -1]], c=[1.0]), -1),  # consumes a non-reactant
    (dict(N=1, M=1, reac=[[0, 0, 1]], stoi=[[0, 0, -2]], c=[1.0]), -1),  # consumes more than it has
    (dict(N=1, M=1, reac=[], stoi=[[0, 2, 1]], c=[1.0]), -1),           # stoichiometry species out of range
])
def test_network_validation_codes(L, case, code):
    rc, msg = _create(L, case["N"], case["M"], case["reac"], case["stoi"], case["c"])
    assert rc == code, (rc, msg)
    assert msg


def test_run_rejects_bad_arguments_on_host(L):
    lib = L.load()
    p = L.rt_run_params()
    o = L.rt_outputs()
    assert lib.rt_run(None, ctypes.byref(p), ctypes.byref(o), None, None, 0, None) == L.RT_ERR_INVALID_ARG
    assert lib.rt_draw_exp1(1, 0, -1, None, None, None, None, None, None) == L.RT_ERR_INVALID_ARG
    assert lib.rt_log_eval(-1, None, None, None) == L.RT_ERR_INVALID_ARG
    assert lib.rt_loglik_backward(None, 1, None, None, None, None, None) == L.RT_ERR_INVALID_ARG
    assert b"NULL" in lib.rt_last_error()


def test_generators_are_deterministic_and_well_formed():
    a = W.random_mass_action(50, 400, seed=9)
    b = W.random_mass_action(50, 400, seed=9)
    for f in ("reac_rxn", "reac_sp", "reac_coef", "stoi_rxn", "stoi_sp", "stoi_delta", "c"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    S = a.dense_reactants()
    V = a.dense_stoich()
    assert S.sum(1).max() <= 2 and S.sum(1).min() >= 1
    assert ((V >= -S)).all()  # consumption only of reactants
    assert (a.c > 0).all()
    items = W.batched_networks(20, seed=3)
    assert len(items) == 20
    for it in items:
        assert it.net.n_species == max(1, it.net.n_reactions // 4)
        assert 1.0 <= it.t_end <= 10.0
        assert it.x0.shape == (it.net.n_species,)


def test_lotka_volterra_is_table_4_model():
    """Table 4: A -> 2A (10), A + B -> 2B (0.01), B -> NULL (10)."""
    net = W.lotka_volterra()
    assert net.dense_reactants().tolist() == [[1, 0], [1, 1], [0, 1]]
    assert net.dense_stoich().tolist() == [[1, 0], [-1, 1], [0, -1]]
    assert net.c.tolist() == [10.0, 0.01, 10.0]


def test_large_network_config_shape_and_realised_dependency_degree():
    """N = 1e4, M = 1e6 with uniform reactants: ~150 reading reactions per species and a dependency
    out-degree of a few hundred per reaction (the recomputes per event of the large-network scan)."""
    net = W.large_network_config()["net"]
    N, M = net.n_species, net.n_reactions
    assert (N, M) == (10_000, 1_000_000)
    pairs = np.unique(np.stack([net.reac_rxn, net.reac_sp], 1), axis=0)
    readers = np.bincount(pairs[:, 1], minlength=N)
    assert 140 < readers.mean() < 160
    changed = net.stoi_delta != 0
    deg = np.bincount(net.stoi_rxn[changed], weights=readers[net.stoi_sp[changed]], minlength=M)
    assert 300 < deg.mean() < 450
