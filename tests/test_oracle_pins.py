"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test fixes part of what the oracle computes with something independent:
published known-answer vectors (Philox), high-precision logarithms (mpmath),
closed-form distributions (Poisson birth-death, binomial isomerisation),
brute-force chemical master equation solutions (dimerisation, small
Lotka-Volterra), the single-step law of the Markov jump process (Eq. 3, 19-23),
exact invariants (Eq. 5), the random-time-change martingale (Eq. 16-18) and the
exact likelihood of a pure-birth path.  All inputs are seeded.

The simulation pins run in both of the oracle's modes: the internal-time form of
Table 2 (every internal time advanced at every event) and the absolute-time form
with the dependency graph (Sec. 5; only the fired channel and the channels reading
a changed species are touched).  Further pins tie the two modes to each other (the
same path up to rounding) and fix the frozen-channel rule of Table 2's note.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg
import scipy.stats

import oracle
from paper_2103_00405_gb300 import workloads as W

MODES = [oracle.MODE_EAGER, oracle.MODE_LAZY, oracle.MODE_RESCALED]


def _run(mode, *args, **kw):
    return oracle.run(*args, mode=mode, **kw)

# ----------------------------------------------------------------------------------
# Random numbers and logarithm
# ----------------------------------------------------------------------------------


def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with Random123 (Salmon et al., SC'11)."""
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert oracle.philox4x32_10(ctr, key).tolist() == want


def _log_inputs():
    rng = np.random.default_rng(7)
    xs = [rng.uniform(0, 1, 3000), np.exp(rng.uniform(-740, 709, 3000)), 1 + rng.uniform(-1e-7, 1e-7, 500),
          1 + rng.uniform(-0.5, 0.5, 1000), (2 * rng.integers(0, 2**52, 2000) + 1) * 2.0**-53]
    edges = [5e-324, 2.2250738585072014e-308, 2.2250738585072009e-308, 1.0, 2.0, 0.5, 1 - 2**-53,
             1 + 2**-52, 1.7976931348623157e308, 2**-53, 1 - 2**-52, math.sqrt(2), math.sqrt(0.5), 3.0, 10.0]
    return np.concatenate(xs + [np.array(edges)])


def test_rt_log_accuracy_against_mpmath():
    """The fixed-point log is within 0.51 ulp of ln x and correctly rounded in >= 99.5% of cases."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 160
    lib = oracle.load()
    worst, miss, n = 0.0, 0, 0
    for x in _log_inputs():
        x = float(x)
        r = lib.oracle_rt_log(x)
        t = mpmath.log(mpmath.mpf(x))
        if x == 1.0:
            assert r == 0.0
            continue
        err = float(abs(mpmath.mpf(r) - t) / math.ulp(float(t)))
        worst = max(worst, err)
        miss += err > 0.5
        n += 1
    assert worst <= 0.51, worst
    assert miss <= 0.005 * n, (miss, n)


def test_rt_log_agrees_with_libm():
    lib = oracle.load()
    for x in _log_inputs():
        x = float(x)
        r, m = lib.oracle_rt_log(x), math.log(x)
        assert abs(r - m) <= 1.0 * math.ulp(m) or r == m, (x, r, m)


def test_uniform_and_exp1_draws():
    """u = (2v+1) 2^-53 from the 52 high bits of (w1:w0) of the right Philox block; E = -ln u ~ Exp(1)."""
    lib = oracle.load()
    seed = 0x1234_5678_9ABC_DEF0
    for (g, k, n, s) in [(0, 0, 0, 0), (5, 3, 1, 0), (2**32 + 7, 11, 10, 4), (123, 0, 2**31 - 1, 9)]:
        out = oracle.philox4x32_10([n >> 1, g & 0xFFFFFFFF, k, s], [seed & 0xFFFFFFFF, seed >> 32])
        w0, w1 = (out[2], out[3]) if n & 1 else (out[0], out[1])
        v = ((int(w1) << 32) | int(w0)) >> 12
        assert lib.oracle_uniform(seed, g, k, n, s) == (2 * v + 1) * 2.0**-53
        e = lib.oracle_exp1(seed, g, k, n, s)
        u = (2 * v + 1) * 2.0**-53
        assert abs(e + math.log(u)) <= math.ulp(e)
    # distribution of many draws
    e = np.array([lib.oracle_exp1(1, j, k, n, 0) for j in range(40) for k in range(10) for n in range(250)])
    assert e.min() > 0
    assert scipy.stats.kstest(e, "expon").pvalue > 1e-4
    assert abs(e.mean() - 1) < 4 / math.sqrt(e.size)


# ----------------------------------------------------------------------------------
# Closed forms and brute-force master equations
# ----------------------------------------------------------------------------------


def _chi2_pvalue(counts, probs, min_expected=5.0):
    """Chi-square GOF with tail pooling so that every bin expects >= min_expected."""
    counts = np.asarray(counts, float)
    probs = np.asarray(probs, float)
    n = counts.sum()
    cb, pb, cur_c, cur_p = [], [], 0.0, 0.0
    for i in range(len(probs)):
        cur_c += counts[i]
        cur_p += probs[i]
        if cur_p * n >= min_expected:
            cb.append(cur_c); pb.append(cur_p); cur_c = cur_p = 0.0
    if cb:
        cb[-1] += cur_c; pb[-1] += cur_p
    cb, pb = np.array(cb), np.array(pb)
    pb = pb / pb.sum()
    stat = ((cb - n * pb) ** 2 / (n * pb)).sum()
    return scipy.stats.chi2.sf(stat, len(cb) - 1)


@pytest.mark.parametrize("mode", MODES)
def test_birth_death_transient_is_poisson(nthreads, mode):
    """0 -> A (k), A -> 0 (gamma A), A(0) = 0: A(t) ~ Poisson(k/gamma (1 - e^{-gamma t}))."""
    net = W.birth_death(100.0, 1.0)
    n_traj = 4000
    o = _run(mode, net, [0], 10.0, n_traj, seed=11, sample_dt=0.25, want_grid=True, n_threads=nthreads)
    assert (o["status"] == oracle.ST_TEND).all()
    for t in (0.25, 1.0, 2.5, 10.0):
        gi = int(round(t / 0.25))
        a = o["grid"][:, gi, 0]
        lam = 100 * (1 - math.exp(-t))
        assert abs(a.mean() - lam) < 4 * math.sqrt(lam / n_traj)
        hist = np.bincount(a, minlength=400)[:400]
        assert _chi2_pvalue(hist, scipy.stats.poisson.pmf(np.arange(400), lam)) > 1e-4


@pytest.mark.parametrize("mode", MODES)
def test_isomerisation_is_binomial(nthreads, mode):
    """A -> B (k1), B -> A (k2), A(0) = n: A(t) ~ Binomial(n, k2/(k1+k2) + k1/(k1+k2) e^{-(k1+k2) t})."""
    k1, k2, n0 = 1.0, 0.5, 50
    net = W.isomerisation(k1, k2)
    n_traj = 20000
    o = _run(mode, net, [n0, 0], 3.0, n_traj, seed=5, sample_dt=0.1, want_grid=True, n_threads=nthreads)
    for t in (0.3, 1.0, 3.0):
        gi = int(round(t / 0.1))
        p = k2 / (k1 + k2) + k1 / (k1 + k2) * math.exp(-(k1 + k2) * t)
        a = o["grid"][:, gi, 0]
        assert (o["grid"][:, gi, 0] + o["grid"][:, gi, 1] == n0).all()
        hist = np.bincount(a, minlength=n0 + 1)
        assert _chi2_pvalue(hist, scipy.stats.binom.pmf(np.arange(n0 + 1), n0, p)) > 1e-4


def _cme_transient(states, rates_fn, p0, times):
    """Solve dp/dt = p Q on an enumerated state space by sparse matrix exponential."""
    index = {s: i for i, s in enumerate(states)}
    rows, cols, vals = [], [], []
    out_rate = np.zeros(len(states))
    for i, s in enumerate(states):
        for nxt, r in rates_fn(s):
            if r <= 0:
                continue
            out_rate[i] += r
            if nxt in index:
                rows.append(i); cols.append(index[nxt]); vals.append(r)
    Q = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(len(states), len(states)))
    Q = Q - scipy.sparse.diags(out_rate)
    res, cur, tprev = [], np.array(p0, float), 0.0
    for t in times:
        cur = scipy.sparse.linalg.expm_multiply(Q.T * (t - tprev), cur)
        tprev = t
        res.append(cur.copy())
    return res


@pytest.mark.parametrize("mode", MODES)
def test_dimerisation_matches_master_equation(nthreads, mode):
    """2A -> B (c1 A(A-1)/2), B -> 2A (c2 B), A0 = 1000: A + 2B = 1000, a 501-state chain."""
    c1, c2 = 0.001, 0.1
    net = W.dimerisation(c1, c2)
    n_traj = 4000
    o = _run(mode, net, [1000, 0], 10.0, n_traj, seed=3, sample_dt=0.1, want_grid=True, n_threads=nthreads)
    assert (o["grid"][:, :, 0] + 2 * o["grid"][:, :, 1] == 1000).all()
    states = list(range(501))

    def rates(b):
        a = 1000 - 2 * b
        return [(b + 1, c1 * a * (a - 1) / 2), (b - 1, c2 * b)]

    p0 = np.zeros(501); p0[0] = 1
    times = [0.1, 1.0, 10.0]
    sol = _cme_transient(states, rates, p0, times)
    for t, p in zip(times, sol):
        b = o["grid"][:, int(round(t / 0.1)), 1]
        hist = np.bincount(b, minlength=501)
        assert _chi2_pvalue(hist, p) > 1e-4
        mean = (p * np.arange(501)).sum()
        sd = math.sqrt((p * (np.arange(501) - mean) ** 2).sum())
        assert abs(b.mean() - mean) < 4 * sd / math.sqrt(n_traj)


@pytest.mark.parametrize("mode", MODES)
def test_small_lotka_volterra_matches_master_equation(nthreads, mode):
    """X -> 2X (c1), X + Y -> 2Y (c2), Y -> 0 (c3) from (10, 10), truncated CME with leak < 1e-9."""
    c1, c2, c3 = 1.0, 0.1, 1.0
    net = W.lotka_volterra(c1, c2, c3)
    n_traj = 20000
    T = 1.0
    o = _run(mode, net, [10, 10], T, n_traj, seed=9, sample_dt=0.5, want_grid=True, n_threads=nthreads)
    cap = 90
    states = [(x, y) for x in range(cap + 1) for y in range(cap + 1)]

    def rates(s):
        x, y = s
        return [((x + 1, y), c1 * x), ((x - 1, y + 1), c2 * x * y), ((x, y - 1), c3 * y)]

    p0 = np.zeros(len(states)); p0[states.index((10, 10))] = 1
    (p,) = _cme_transient(states, rates, p0, [T])
    assert 1 - p.sum() < 1e-9  # probability that leaked out of the box
    gx = o["grid"][:, 2, 0]
    gy = o["grid"][:, 2, 1]
    assert gx.max() <= cap and gy.max() <= cap
    P = p.reshape(cap + 1, cap + 1)
    hx = np.bincount(gx, minlength=cap + 1)
    hy = np.bincount(gy, minlength=cap + 1)
    assert _chi2_pvalue(hx, P.sum(1)) > 1e-4
    assert _chi2_pvalue(hy, P.sum(0)) > 1e-4
    joint = np.bincount(gx * (cap + 1) + gy, minlength=(cap + 1) ** 2)
    assert _chi2_pvalue(joint, p, min_expected=20) > 1e-4


@pytest.mark.parametrize("mode", MODES)
def test_single_step_law(nthreads, mode):
    """First event: waiting time ~ Exp(sum a), channel k with probability a_k / sum a, independent (Eq. 3, 23, 26)."""
    net = W.random_mass_action(5, 7, seed=101, c_sigma=0.7)
    x0 = np.array([4, 9, 2, 6, 3], np.int32)
    n_traj = 30000
    o = _run(mode, net, x0, math.inf, n_traj, seed=2, max_events=1, trace_len=1, n_threads=nthreads)
    mu, dt = o["trace_mu"][:, 0], o["trace_t"][:, 0]
    S, V = net.dense_reactants(), net.dense_stoich()
    a = np.array([net.c[k] * np.prod([math.comb(int(x0[i]), int(S[k, i])) for i in range(5)]) for k in range(7)])
    assert (mu >= 0).all()
    assert scipy.stats.kstest(dt, "expon", args=(0, 1 / a.sum())).pvalue > 1e-4
    assert _chi2_pvalue(np.bincount(mu, minlength=7), a / a.sum()) > 1e-4
    # independence of channel and waiting time
    med = np.median(dt)
    table = np.stack([np.bincount(mu[dt < med], minlength=7), np.bincount(mu[dt >= med], minlength=7)])
    table = table[:, table.sum(0) > 0]
    assert scipy.stats.chi2_contingency(table)[1] > 1e-4
    # state after the first event is X0 + v_mu (Eq. 5)
    assert (o["x_final"] == x0 + V[mu]).all()


@pytest.mark.parametrize("mode", MODES)
def test_linear_network_mean_solves_the_rate_equation(nthreads, mode):
    """First-order network: E[X(t)] solves dm/dt = J m + b exactly (matrix exponential)."""
    # 0 -> A (5), A -> B (1), B -> A (0.5), B -> 0 (0.3), A -> 0 (0.2)
    net = W._from_lists(2, [({}, {0: 1}, 5.0), ({0: 1}, {1: 1}, 1.0), ({1: 1}, {0: 1}, 0.5),
                            ({1: 1}, {}, 0.3), ({0: 1}, {}, 0.2)], "linear")
    J = np.array([[-1.2, 0.5], [1.0, -0.8]])
    b = np.array([5.0, 0.0])
    m0 = np.array([3.0, 7.0])
    n_traj = 20000
    o = _run(mode, net, m0.astype(np.int32), 3.0, n_traj, seed=4, sample_dt=1.0, want_grid=True, n_threads=nthreads)
    aug = np.zeros((3, 3)); aug[:2, :2] = J; aug[:2, 2] = b
    for gi, t in enumerate([0.0, 1.0, 2.0, 3.0]):
        m = (scipy.linalg.expm(aug * t) @ np.append(m0, 1.0))[:2]
        X = o["grid"][:, gi, :].astype(float)
        se = X.std(0) / math.sqrt(n_traj) + 1e-12
        assert (np.abs(X.mean(0) - m) < 4 * se + 1e-12).all(), (t, X.mean(0), m)


# ----------------------------------------------------------------------------------
# Exact relations
# ----------------------------------------------------------------------------------


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_state_equals_initial_plus_counts_times_stoichiometry(seed, nthreads, mode):
    """X(t) = X(0) + sum_k n_k v_k exactly (Eq. 5), for every trajectory."""
    net = W.random_mass_action(6, 12, seed=200 + seed)
    x0 = W.poisson_x0(6, 20, seed)
    o = _run(mode, net, x0, 2.0, 200, seed=seed, max_events=20000, want_grad=True, n_threads=nthreads)
    V = net.dense_stoich()
    assert (o["x_final"] == x0 + o["counts"].astype(np.int64) @ V).all()
    assert (o["n_events"] == o["counts"].sum(1)).all()


@pytest.mark.parametrize("mode", MODES)
def test_grid_is_right_continuous_state_from_event_trace(mode):
    """Grid value at g = X0 + sum of v_mu over events with time <= g, rebuilt from the event trace."""
    net = W.lotka_volterra()
    x0 = np.array([1000, 1000], np.int32)
    o = _run(mode, net, x0, 0.05, 8, seed=1, sample_dt=0.001, want_grid=True, trace_len=5000)
    V = net.dense_stoich()
    G = o["grid"].shape[1]
    for j in range(8):
        n = int(o["n_events"][j])
        assert n < 5000
        mu, tt = o["trace_mu"][j, :n], o["trace_t"][j, :n]
        assert (np.diff(tt) >= 0).all()
        cum = x0 + np.concatenate([[np.zeros(2, np.int64)], np.cumsum(V[mu], 0)])
        for gi in range(G):
            g = gi * 0.001
            m = np.searchsorted(tt, g, side="right")
            assert (o["grid"][j, gi] == cum[m]).all()


@pytest.mark.parametrize("mode", MODES)
def test_internal_time_martingale(nthreads, mode):
    """n_k(t) - T_k(t) is a martingale with mean 0 (random time change, Eq. 16-18)."""
    net = W.random_mass_action(4, 8, seed=77, c_sigma=0.5)
    x0 = W.poisson_x0(4, 30, 78)
    n_traj = 20000
    o = _run(mode, net, x0, 1.0, n_traj, seed=6, want_grad=True, max_events=100000, n_threads=nthreads)
    ok = o["status"] == oracle.ST_TEND
    assert ok.mean() > 0.99
    d = o["counts"][ok] - o["t_internal"][ok]
    se = d.std(0) / math.sqrt(ok.sum()) + 1e-12
    assert (np.abs(d.mean(0)) < 4 * se).all()


@pytest.mark.parametrize("mode", MODES)
def test_pure_birth_likelihood_and_gradient(mode):
    """0 -> A at rate c on [0, t]: l = n ln c - c t and dl/dc = n/c - t."""
    c, T = 2.5, 3.0
    net = W.pure_birth(c)
    o = _run(mode, net, [0], T, 50, seed=3, want_grad=True)
    n = o["counts"][:, 0].astype(float)
    assert (o["x_final"][:, 0] == n).all()
    np.testing.assert_allclose(o["t_internal"][:, 0], c * T, rtol=1e-13)
    np.testing.assert_allclose(o["loglik"], n * math.log(c) - c * T, rtol=1e-12, atol=1e-12)
    g = oracle.loglik_backward(np.ones(50), o["counts"], o["t_internal"], net.c)
    np.testing.assert_allclose(g[0], (n / c - T).sum(), rtol=1e-11)


@pytest.mark.parametrize("mode", MODES)
def test_loglik_matches_path_integral_from_trace(mode):
    """l = sum over events of ln a_mu(X before) - integral of sum_k a_k(X(s)) ds, rebuilt from the trace."""
    net = W.random_mass_action(4, 6, seed=31, c_sigma=0.5)
    x0 = np.array([15, 12, 9, 20], np.int32)
    T = 0.5
    o = _run(mode, net, x0, T, 6, seed=8, want_grad=True, trace_len=20000)
    S, V = net.dense_reactants(), net.dense_stoich()

    def props(x):
        return np.array([net.c[k] * np.prod([math.comb(int(x[i]), int(S[k, i])) for i in range(4)])
                         for k in range(6)])

    for j in range(6):
        assert o["status"][j] == oracle.ST_TEND
        n = int(o["n_events"][j])
        x = x0.astype(np.int64).copy()
        t, ll, integ = 0.0, 0.0, np.zeros(6)
        for e in range(n):
            mu, te = o["trace_mu"][j, e], o["trace_t"][j, e]
            a = props(x)
            integ += a * (te - t)
            ll += math.log(a[mu])
            x += V[mu]
            t = te
        integ += props(x) * (T - t)
        np.testing.assert_allclose(o["t_internal"][j], integ, rtol=1e-9)
        np.testing.assert_allclose(o["loglik"][j], ll - integ.sum(), rtol=1e-9, atol=1e-9)


def _path_loglik(net, x0, T, mu, tt, c):
    """l(c; path) = sum ln(c_mu h_mu(X before)) - sum_k c_k int h_k dt for a fixed recorded path."""
    S, V = net.dense_reactants(), net.dense_stoich()
    M, N = S.shape
    x = x0.astype(np.int64).copy()
    t, ll, ih = 0.0, 0.0, np.zeros(M)
    for m, te in zip(mu, tt):
        h = np.array([np.prod([math.comb(int(x[i]), int(S[k, i])) for i in range(N)]) for k in range(M)], float)
        ih += h * (te - t)
        ll += math.log(c[m] * h[m])
        x += V[m]
        t = te
    h = np.array([np.prod([math.comb(int(x[i]), int(S[k, i])) for i in range(N)]) for k in range(M)], float)
    ih += h * (T - t)
    return ll - (c * ih).sum()


@pytest.mark.parametrize("mode", MODES)
def test_gradient_against_fixed_path_finite_differences(mode):
    """d l/d c_k = (n_k - T_k(t_end)) / c_k against central differences of the recorded path's likelihood."""
    net = W.random_mass_action(3, 5, seed=55, c_sigma=0.4)
    x0 = np.array([10, 8, 12], np.int32)
    T, n_traj = 0.3, 12
    o = _run(mode, net, x0, T, n_traj, seed=12, want_grad=True, trace_len=4000)
    g = (o["counts"] - o["t_internal"]) / net.c
    for j in range(n_traj):
        n = int(o["n_events"][j])
        mu, tt = o["trace_mu"][j, :n], o["trace_t"][j, :n]
        np.testing.assert_allclose(_path_loglik(net, x0, T, mu, tt, net.c), o["loglik"][j], rtol=1e-10)
        for k in range(net.n_reactions):
            h = 1e-6 * net.c[k]
            cp, cm = net.c.copy(), net.c.copy()
            cp[k] += h
            cm[k] -= h
            fd = (_path_loglik(net, x0, T, mu, tt, cp) - _path_loglik(net, x0, T, mu, tt, cm)) / (cp[k] - cm[k])
            scale = max(abs(g[j, k]), o["counts"][j, k] / net.c[k], 1.0)
            assert abs(fd - g[j, k]) <= 1e-6 * scale, (j, k, fd, g[j, k])


def test_score_is_the_likelihood_ratio_derivative_under_common_random_numbers(nthreads):
    """E[f(X) dl/dc_k] = d E[f(X)] / d c_k; the right side by central differences of runs at c +- h that
    share every random number (the random-time coupling: same seed, same per-channel Exp(1) streams)."""
    net = W.random_mass_action(3, 5, seed=55, c_sigma=0.4)
    x0 = np.array([10, 8, 12], np.int32)
    T, n_traj = 0.5, 40000
    base = oracle.run(net, x0, T, n_traj, seed=21, want_grad=True, n_threads=nthreads)
    score = (base["counts"] - base["t_internal"]) / net.c
    f = base["x_final"].astype(float)
    for k in range(net.n_reactions):
        h = 0.02 * net.c[k]
        cp, cm = net.c.copy(), net.c.copy()
        cp[k] += h
        cm[k] -= h
        fp = oracle.run(net.with_rates(cp), x0, T, n_traj, seed=21, n_threads=nthreads)["x_final"].astype(float)
        fm = oracle.run(net.with_rates(cm), x0, T, n_traj, seed=21, n_threads=nthreads)["x_final"].astype(float)
        fd = (fp - fm) / (2 * h)
        lr = f * score[:, k:k + 1]
        for i in range(3):
            se = math.sqrt(fd[:, i].var() / n_traj + lr[:, i].var() / n_traj)
            assert abs(fd[:, i].mean() - lr[:, i].mean()) < 4 * se + 1e-9, (k, i)


@pytest.mark.parametrize("mode", MODES)
def test_absorbing_overflow_bad_x0_and_event_cap(mode):
    """Status semantics: absorption, int32 overflow (event not fired), negative X0, max_events."""
    death = W._from_lists(1, [({0: 1}, {}, 1.0)], "death")
    o = _run(mode, death, [5], math.inf, 3, seed=1)
    assert (o["status"] == oracle.ST_ABSORBED).all() and (o["x_final"] == 0).all() and (o["n_events"] == 5).all()
    birth = W.pure_birth(1e6)
    o = _run(mode, birth, [2**31 - 3], math.inf, 2, seed=1)
    assert (o["status"] == oracle.ST_OVERFLOW).all() and (o["x_final"][:, 0] == 2**31 - 1).all()
    o = _run(mode, W.birth_death(), np.array([[-1], [3]], np.int32), 1.0, 2, seed=1, want_grad=True)
    assert o["status"].tolist() == [oracle.ST_BAD_X0, oracle.ST_TEND] and math.isnan(o["loglik"][0])
    o = _run(mode, W.lotka_volterra(), [1000, 1000], 10.0, 2, seed=1, max_events=100)
    assert (o["status"] == oracle.ST_MAX_EVENTS).all() and (o["n_events"] == 100).all()
    o = _run(mode, W.lotka_volterra(), [1000, 1000], 10.0, 2, seed=1, max_events=0)
    assert (o["status"] == oracle.ST_MAX_EVENTS).all() and (o["x_final"] == 1000).all()
    o = _run(mode, W.lotka_volterra(), [1000, 1000], 0.0, 2, seed=1, sample_dt=0.1, want_grid=True)
    assert (o["status"] == oracle.ST_TEND).all() and o["grid"].shape == (2, 1, 2) and (o["n_events"] == 0).all()


def test_grid_length_rule():
    assert oracle.grid_len(5.0, 0.01) == 501
    assert oracle.grid_len(10.0, 0.01) == 1001
    assert oracle.grid_len(1.0, 0.3) == 4
    assert oracle.grid_len(1.0, 0.0) == 0
    assert oracle.grid_len(math.inf, 0.1) == 0


# ----------------------------------------------------------------------------------
# The absolute-time form against the internal-time form, and frozen channels
# ----------------------------------------------------------------------------------


@pytest.mark.parametrize("mode", [oracle.MODE_LAZY, oracle.MODE_RESCALED])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_other_forms_follow_the_same_path_as_table_2(seed, mode, nthreads):
    """The absolute-time form and Table 3's rescaled form are the same method as Table 2's
    internal-time form in exact arithmetic: on random uni/bimolecular networks the event streams
    agree (channel by channel) and the times to within rounding, as long as no two channels are
    within rounding of a tie.  A channel left stale (not touched although it reads a changed
    species, its internal time not brought up to the event, a waiting time not rescaled, a
    frozen remaining internal time lost) changes the path within a few events."""
    net = W.random_mass_action(8, 40, seed=300 + seed, c_sigma=0.8)
    x0 = W.poisson_x0(8, 25, seed)
    K = 400
    e = oracle.run(net, x0, math.inf, 64, seed=seed, max_events=K, want_grad=True, trace_len=K, n_threads=nthreads)
    z = oracle.run(net, x0, math.inf, 64, seed=seed, max_events=K, want_grad=True, trace_len=K, n_threads=nthreads,
                   mode=mode)
    same = (e["trace_mu"] == z["trace_mu"]).all(1)
    assert same.mean() >= 0.95, same.mean()
    assert (e["trace_mu"][:, 0] == z["trace_mu"][:, 0]).all()  # the first event is computed identically
    assert (e["trace_t"][:, 0] == z["trace_t"][:, 0]).all()
    np.testing.assert_allclose(z["trace_t"][same], e["trace_t"][same], rtol=1e-10, atol=0)
    assert (z["x_final"][same] == e["x_final"][same]).all() and (z["counts"][same] == e["counts"][same]).all()
    np.testing.assert_allclose(z["t_internal"][same], e["t_internal"][same], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(z["loglik"][same], e["loglik"][same], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("mode", MODES)
def test_forbidden_channel_is_frozen(mode, nthreads):
    """Table 2's note: a channel forbidden to fire keeps a frozen internal time.  Birth-death with
    its death channel forbidden is a pure birth process, A(t) ~ Poisson(k t); and forbidding a
    channel is the same, bit for bit, as giving it rate 0."""
    net = W.birth_death(20.0, 1.0)
    o = _run(mode, net, [0], 2.0, 6000, seed=4, want_grad=True, enabled=[1, 0], n_threads=nthreads)
    assert (o["counts"][:, 1] == 0).all() and (o["t_internal"][:, 1] == 0).all()
    a = o["x_final"][:, 0]
    assert abs(a.mean() - 40.0) < 4 * math.sqrt(40.0 / 6000)
    assert _chi2_pvalue(np.bincount(a, minlength=120)[:120], scipy.stats.poisson.pmf(np.arange(120), 40.0)) > 1e-4
    rnet = W.random_mass_action(5, 10, seed=41)
    x0 = W.poisson_x0(5, 30, 42)
    en = np.array([1, 1, 0, 1, 0, 1, 1, 1, 0, 1], np.uint8)
    c0 = rnet.c * en
    f = _run(mode, rnet, x0, 0.5, 20, seed=2, want_grad=True, trace_len=300, enabled=en, n_threads=nthreads)
    z = _run(mode, rnet.with_rates(c0), x0, 0.5, 20, seed=2, want_grad=True, trace_len=300, n_threads=nthreads)
    for k in ("x_final", "n_events", "counts", "trace_mu"):
        assert np.array_equal(f[k], z[k]), k
    for k in ("t_last", "t_internal", "loglik", "trace_t"):
        assert np.array_equal(f[k].view(np.int64), z[k].view(np.int64)), k
    assert (f["counts"][:, en == 0] == 0).all()


@pytest.mark.parametrize("mode", MODES)
def test_frozen_channel_resumes_with_its_remaining_internal_time(mode):
    """A channel whose propensity drops to 0 and comes back keeps its unused internal time
    (Table 2's refresh rule; Table 3 with the frozen-channel reading): A -> B, B -> A at rates
    making the reverse channel switch on and off, against Table 2's form event by event."""
    net = W.isomerisation(3.0, 1.0)
    e = oracle.run(net, [1, 0], 20.0, 200, seed=7, trace_len=400)
    z = _run(mode, net, [1, 0], 20.0, 200, seed=7, trace_len=400)
    assert (e["trace_mu"] == z["trace_mu"]).mean() > 0.99
    np.testing.assert_allclose(z["trace_t"], e["trace_t"], rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------------
# Time-dependent rates c_k(t) = c_k (1 + beta_k t)  (Sec. 6, Eq. 29)
# ----------------------------------------------------------------------------------


def test_zero_slopes_reproduce_constant_rates_bit_for_bit(nthreads):
    net = W.random_mass_action(5, 9, seed=401)
    x0 = W.poisson_x0(5, 20, 402)
    a = oracle.run(net, x0, 1.0, 50, seed=3, want_grad=True, want_grid=True, sample_dt=0.1, trace_len=300,
                   n_threads=nthreads)
    b = oracle.run(net, x0, 1.0, 50, seed=3, want_grad=True, want_grid=True, sample_dt=0.1, trace_len=300,
                   n_threads=nthreads, beta=np.zeros(9))
    for k in a:
        assert np.array_equal(a[k].view(np.int64) if a[k].dtype == np.float64 else a[k],
                              b[k].view(np.int64) if b[k].dtype == np.float64 else b[k]), k


def test_ramped_birth_is_poisson_with_the_integrated_rate(nthreads):
    """0 -> A at c (1 + beta t): A(t) ~ Poisson(c (t + beta t^2 / 2))."""
    c, beta, n = 20.0, 0.7, 20000
    o = oracle.run(W.pure_birth(c), [0], 3.0, n, seed=8, sample_dt=0.5, want_grid=True, beta=[beta],
                   n_threads=nthreads)
    for gi, t in ((1, 0.5), (4, 2.0), (6, 3.0)):
        lam = c * (t + beta * t * t / 2)
        x = o["grid"][:, gi, 0]
        assert abs(x.mean() - lam) < 4 * math.sqrt(lam / n)
        top = int(lam + 10 * math.sqrt(lam)) + 10
        assert _chi2_pvalue(np.bincount(x, minlength=top)[:top], scipy.stats.poisson.pmf(np.arange(top), lam)) > 1e-4


def test_birth_death_with_ramped_immigration_solves_the_mean_equation(nthreads):
    """0 -> A at k (1 + beta t), A -> 0 at gamma A, A(0) = 0: A(t) is Poisson with mean
    m(t) = k/g - k b/g^2 + (k b / g) t - (k/g - k b/g^2) e^{-g t}."""
    k, g, beta, n = 50.0, 1.0, 0.5, 20000
    o = oracle.run(W.birth_death(k, g), [0], 4.0, n, seed=12, sample_dt=1.0, want_grid=True, beta=[beta, 0.0],
                   n_threads=nthreads)
    for gi in (1, 2, 4):
        t = float(gi)
        m = k / g - k * beta / g ** 2 + (k * beta / g) * t - (k / g - k * beta / g ** 2) * math.exp(-g * t)
        x = o["grid"][:, gi, 0]
        assert abs(x.mean() - m) < 4 * math.sqrt(m / n)
        top = int(m + 10 * math.sqrt(m)) + 10
        assert _chi2_pvalue(np.bincount(x, minlength=top)[:top], scipy.stats.poisson.pmf(np.arange(top), m)) > 1e-4


def test_first_event_law_with_ramped_rates(nthreads):
    """First event from t = 0: P(tau > s) = exp(-sum_k A_k (s + beta_k s^2 / 2)), channel k with
    probability a_k(tau) / sum a(tau) given tau."""
    net = W.random_mass_action(4, 6, seed=77, c_sigma=0.5)
    x0 = np.array([6, 9, 4, 7], np.int32)
    beta = np.array([0.0, 2.0, 5.0, 0.5, 1.0, 3.0])
    n = 30000
    o = oracle.run(net, x0, math.inf, n, seed=5, max_events=1, trace_len=1, beta=beta, n_threads=nthreads)
    S = net.dense_reactants()
    A = np.array([net.c[k] * np.prod([math.comb(int(x0[i]), int(S[k, i])) for i in range(4)]) for k in range(6)])
    tau = o["trace_t"][:, 0]
    cdf = lambda s: 1 - np.exp(-(A.sum() * s + (A * beta).sum() * s * s / 2))
    assert scipy.stats.kstest(tau, cdf).pvalue > 1e-4
    # channel given the time: probabilities proportional to A_k (1 + beta_k tau); chi-square on the
    # expected counts summed over the observed times
    mu = o["trace_mu"][:, 0]
    p = A[None, :] * (1 + beta[None, :] * tau[:, None])
    p /= p.sum(1, keepdims=True)
    assert _chi2_pvalue(np.bincount(mu, minlength=6), p.sum(0) / n) > 1e-4


@pytest.mark.parametrize("seed", [1, 2])
def test_ramped_internal_times_and_likelihood_from_the_trace(seed):
    """T_k(t_end) = int_0^T c_k (1 + beta_k s) h_k(X(s)) ds and l = sum ln a_mu(t_mu) - sum_k T_k,
    rebuilt from the event trace with the closed-form integral of each step."""
    net = W.random_mass_action(4, 6, seed=31 + seed, c_sigma=0.5)
    x0 = np.array([15, 12, 9, 20], np.int32)
    beta = np.array([0.0, 1.5, 0.3, 2.0, 0.0, 0.8])
    T = 0.5
    o = oracle.run(net, x0, T, 6, seed=8, want_grad=True, trace_len=20000, beta=beta)
    S, V = net.dense_reactants(), net.dense_stoich()

    def hvec(x):
        return np.array([np.prod([math.comb(int(x[i]), int(S[k, i])) for i in range(4)]) for k in range(6)], float)

    for j in range(6):
        n = int(o["n_events"][j])
        x = x0.astype(np.int64).copy()
        t, ll, integ = 0.0, 0.0, np.zeros(6)
        for e in range(n):
            mu, te = o["trace_mu"][j, e], o["trace_t"][j, e]
            h = hvec(x)
            integ += net.c * h * ((te - t) + beta * (te * te - t * t) / 2)
            ll += math.log(net.c[mu] * h[mu] * (1 + beta[mu] * te))
            x += V[mu]
            t = te
        integ += net.c * hvec(x) * ((T - t) + beta * (T * T - t * t) / 2)
        np.testing.assert_allclose(o["t_internal"][j], integ, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(o["loglik"][j], ll - integ.sum(), rtol=1e-9, atol=1e-9)
