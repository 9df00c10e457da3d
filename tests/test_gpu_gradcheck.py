"""Gradient checks of the GPU path at the gradient workload's size (M = 64, N = 16,
c ~ lognormal(0, 0.5), X0 ~ Poisson(200), 65536 trajectories to t_end = 5), through the C ABI.

The score of the path log-likelihood (Eq. 16-18) is dl/dc_k = n_k / c_k - int h_k dt, and the
GPU returns it as (n_k - T_k(t_end)) / c_k.  Three checks:
  * fixed path: int h_k dt rebuilt in numpy from the GPU's own event trace (the recorded
    states and event times) and the central difference of the recorded path's likelihood
    at c +- 1e-6 c_k (channel k's term of the separable sum), against the GPU's score,
    within 1e-6 relative (scale floor n_k / c_k);
  * likelihood ratio: d E[f] / d c_k = E[f score_k] for f = the final state, the left side by
    central differences of runs that share every random number (common random numbers: the
    same seed, so the same unit Poisson process per channel, Eq. 16), within 4 standard errors;
  * re-simulation (a reported diagnostic): at c +- 1e-6 c_k with the same random numbers, the
    fraction of trajectories whose event stream is unchanged, and for those the relative gap
    between the re-simulated difference quotient of the likelihood and the score (they are
    not equal: moving c moves the event times, so the quotient is a total derivative).
"""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_00405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_2103_00405_gb300 import api  # noqa: E402
from paper_2103_00405_gb300 import build as B  # noqa: E402

B.build()

CFG = W.grad_config()
NET = CFG["net"]
M, N = NET.n_reactions, NET.n_species


def _h(x):
    """h_k(x) for every channel from the dense reactant matrix (Eq. 2)."""
    S = NET.dense_reactants()
    out = np.ones(M)
    for i in range(N):
        for k in np.flatnonzero(S[:, i]):
            out[k] *= math.comb(int(x[i]), int(S[k, i]))
    return out


def test_fixed_path_finite_differences_against_the_gpu_score():
    n = 65536
    K = 8000
    netg = api.Network(NET)
    full = api.simulate(netg, CFG["x0"], CFG["t_end"], n, seed=1, max_events=10**8, grad=True)
    torch.cuda.synchronize()
    counts = full["counts"].cpu().numpy()
    Tend = full["t_internal"].cpu().numpy()
    V = NET.dense_stoich()
    c = NET.c
    for j in (0, 1, 777, 40000, 65535):
        # the same trajectory (same global id) alone, with its event trace
        g = api.simulate(netg, CFG["x0"], CFG["t_end"], 1, seed=1, traj_offset=j, max_events=10**8, grad=True,
                         trace_len=K)
        ev = int(g["n_events"][0].item())
        assert ev < K and ev == int(full["n_events"][j].item())
        assert np.array_equal(g["counts"][0].cpu().numpy(), counts[j])
        assert np.array_equal(g["t_internal"][0].cpu().numpy().view(np.int64), Tend[j].view(np.int64))
        mu = g["trace_mu"][0, :ev].cpu().numpy()
        tt = g["trace_t"][0, :ev].cpu().numpy()
        x = CFG["x0"].astype(np.int64).copy()
        H = np.zeros(M)  # int h_k dt along the recorded path
        tprev = 0.0
        for m, te in zip(mu, tt):
            H += _h(x) * (te - tprev)
            x += V[m]
            tprev = te
        H += _h(x) * (CFG["t_end"] - tprev)
        assert np.array_equal(x, full["x_final"][j].cpu().numpy())
        nk = np.bincount(mu, minlength=M)
        assert np.array_equal(nk, counts[j])

        # the recorded path's log-likelihood is separable in c: l(c) = sum_k (n_k ln c_k - c_k H_k) + sum ln h_mu,
        # so the central difference in c_k involves channel k's term only (differencing the whole sum
        # would cancel ~1e4 against a step of ~1e-6)
        def path_ll_k(k, ck):
            return nk[k] * math.log(ck) - ck * H[k]

        score = (counts[j] - Tend[j]) / c
        for k in range(M):
            hk = 1e-6 * c[k]
            cp, cm = c[k] + hk, c[k] - hk
            fd = (path_ll_k(k, cp) - path_ll_k(k, cm)) / (cp - cm)
            scale = max(abs(score[k]), counts[j, k] / c[k], 1.0)
            assert abs(fd - score[k]) <= 1e-6 * scale, (j, k, fd, score[k])


def test_likelihood_ratio_identity_at_full_size():
    """d E[X_final] / d c_k = E[X_final * score_k] for the four most active channels."""
    n = 65536
    netg = api.Network(NET)
    base = api.simulate(netg, CFG["x0"], CFG["t_end"], n, seed=3, max_events=10**8, grad=True)
    counts = base["counts"].cpu().numpy()
    score = (counts - base["t_internal"].cpu().numpy()) / NET.c
    f = base["x_final"].cpu().numpy().astype(float)
    for k in np.argsort(-counts.sum(0))[:4]:
        hk = 0.05 * NET.c[k]
        cp, cm = NET.c.copy(), NET.c.copy()
        cp[k] += hk
        cm[k] -= hk
        fp = api.simulate(api.Network(NET, cp), CFG["x0"], CFG["t_end"], n, seed=3, max_events=10**8)
        fm = api.simulate(api.Network(NET, cm), CFG["x0"], CFG["t_end"], n, seed=3, max_events=10**8)
        fd = (fp["x_final"].cpu().numpy().astype(float) - fm["x_final"].cpu().numpy().astype(float)) / (2 * hk)
        lr = f * score[:, k:k + 1]
        for i in range(N):
            se = math.sqrt(fd[:, i].var() / n + lr[:, i].var() / n)
            assert abs(fd[:, i].mean() - lr[:, i].mean()) < 4 * se + 1e-9, (k, i, fd[:, i].mean(), lr[:, i].mean())


def test_common_random_number_resimulation_diagnostic(capsys):
    n = 65536
    netg = api.Network(NET)
    base = api.simulate(netg, CFG["x0"], CFG["t_end"], n, seed=1, max_events=10**8, grad=True)
    counts = base["counts"].cpu().numpy()
    score = (counts - base["t_internal"].cpu().numpy()) / NET.c
    rows = []
    for k in np.argsort(-counts.sum(0))[:3]:
        hk = 1e-6 * NET.c[k]
        cp, cm = NET.c.copy(), NET.c.copy()
        cp[k] += hk
        cm[k] -= hk
        op = api.simulate(api.Network(NET, cp), CFG["x0"], CFG["t_end"], n, seed=1, max_events=10**8, grad=True)
        om = api.simulate(api.Network(NET, cm), CFG["x0"], CFG["t_end"], n, seed=1, max_events=10**8, grad=True)
        same = np.ones(n, bool)
        for o in (op, om):
            same &= (o["counts"].cpu().numpy() == counts).all(1)
            same &= (o["x_final"].cpu().numpy() == base["x_final"].cpu().numpy()).all(1)
        fd = (op["loglik"].cpu().numpy() - om["loglik"].cpu().numpy()) / (cp[k] - cm[k])
        scale = np.maximum(np.abs(score[:, k]), counts[:, k] / NET.c[k])
        gap = np.abs(fd - score[:, k])[same] / np.maximum(scale[same], 1.0)
        rows.append(dict(channel=int(k), unchanged_fraction=float(same.mean()),
                         median_relative_gap=float(np.median(gap)) if gap.size else None,
                         max_relative_gap=float(gap.max()) if gap.size else None))
        assert np.isfinite(fd).all() and 0.0 < same.mean() <= 1.0
    with capsys.disabled():
        print("\ncommon-random-number re-simulation at c +- 1e-6 c_k:", json.dumps(rows))
