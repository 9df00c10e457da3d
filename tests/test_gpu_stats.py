"""Ensemble statistics of GPU runs against closed forms, at the benchmarked ensemble size.

Parity tests show that the CUDA path reproduces the oracle's trajectories bit for bit; these
tests check the laws themselves on 2^20 GPU trajectories per network through the ensemble
moments output (exact integer sums of X and X^2 per grid point): the mean and the variance at
every grid time must lie within 4 standard errors of the exact values.

* birth-death, 0 -> A (k), A -> 0 (gamma A), A0 = 0: A(t) ~ Poisson(k/gamma (1 - e^{-gamma t}));
* isomerisation, A -> B (k1 A), B -> A (k2 B), A0 = n: A(t) ~ Binomial(n, p(t)),
  p(t) = k2/(k1+k2) + k1/(k1+k2) e^{-(k1+k2) t};
* dimerisation, 2A -> B (c1 A(A-1)/2), B -> 2A (c2 B), A0 = 1000: A + 2B = 1000 is conserved, so
  the law of B(t) solves the master equation of a 501-state chain, here by a matrix exponential.

Standard errors: sd / sqrt(n) for the mean and sqrt((mu4 - sd^4) / n) for the variance, with the
exact fourth central moment of each law.
"""
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

N_TRAJ = 1 << 20
T_END = 10.0
DT = 1.0


def _moments(net, x0, seed):
    g = api.simulate(api.Network(net), x0, T_END, N_TRAJ, seed=seed, sample_dt=DT, grid="moments",
                     max_events=W.ENSEMBLE_MAX_EVENTS)
    torch.cuda.synchronize()
    assert (g["status"] == 0).all()
    n = g["grid_count"].cpu().numpy().astype(np.float64)
    s = g["grid_sum"].cpu().numpy().astype(np.float64)
    q = g["grid_sumsq"].cpu().numpy().astype(np.float64)
    assert (n == N_TRAJ).all()
    mean = s / n[:, None]
    var = (q - s * s / n[:, None]) / (n[:, None] - 1)
    return mean, var


def _check(mean, var, mu, sd2, mu4, what):
    se_mean = math.sqrt(sd2 / N_TRAJ)
    se_var = math.sqrt(max(mu4 - sd2 * sd2, 0.0) / N_TRAJ)
    assert abs(mean - mu) <= 4 * se_mean, (what, mean, mu, se_mean)
    assert abs(var - sd2) <= 4 * se_var, (what, var, sd2, se_var)


def test_birth_death_ensemble_is_poisson():
    k, gamma = 100.0, 1.0
    mean, var = _moments(W.birth_death(k, gamma), np.array([0], np.int32), seed=11)
    assert mean[0, 0] == 0 and var[0, 0] == 0
    for i in range(1, mean.shape[0]):
        lam = k / gamma * (1.0 - math.exp(-gamma * i * DT))
        _check(mean[i, 0], var[i, 0], lam, lam, lam * (1.0 + 3.0 * lam), ("birth-death", i))


def test_isomerisation_ensemble_is_binomial():
    k1, k2, n0 = 1.0, 0.5, 200
    mean, var = _moments(W.isomerisation(k1, k2), np.array([n0, 0], np.int32), seed=12)
    for i in range(1, mean.shape[0]):
        t = i * DT
        p = k2 / (k1 + k2) + k1 / (k1 + k2) * math.exp(-(k1 + k2) * t)
        s2 = n0 * p * (1 - p)
        mu4 = s2 * (1 + 3 * (n0 - 2) * p * (1 - p))
        _check(mean[i, 0], var[i, 0], n0 * p, s2, mu4, ("isomerisation A", i))
        _check(mean[i, 1], var[i, 1], n0 * (1 - p), s2, mu4, ("isomerisation B", i))


def test_dimerisation_ensemble_matches_master_equation():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    c1, c2 = 0.001, 0.1
    mean, var = _moments(W.dimerisation(c1, c2), np.array([1000, 0], np.int32), seed=13)
    # generator of B on {0..500}: B -> B + 1 at c1 A (A - 1) / 2, B -> B - 1 at c2 B, A = 1000 - 2 B
    Q = np.zeros((501, 501))
    for b in range(501):
        a = 1000 - 2 * b
        up, down = c1 * a * (a - 1) / 2, c2 * b
        if b < 500:
            Q[b, b + 1] = up
        if b > 0:
            Q[b, b - 1] = down
        Q[b, b] = -(up if b < 500 else 0.0) - down
    p0 = np.zeros(501)
    p0[0] = 1.0
    step = scipy_linalg.expm(Q * DT)
    p = p0
    states = np.arange(501, dtype=np.float64)
    for i in range(1, mean.shape[0]):
        p = p @ step
        mu = float((p * states).sum())
        s2 = float((p * (states - mu) ** 2).sum())
        mu4 = float((p * (states - mu) ** 4).sum())
        _check(mean[i, 1], var[i, 1], mu, s2, mu4, ("dimerisation B", i))
        # A = 1000 - 2 B exactly
        _check(mean[i, 0], var[i, 0], 1000 - 2 * mu, 4 * s2, 16 * mu4, ("dimerisation A", i))
