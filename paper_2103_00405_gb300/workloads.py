"""Seeded synthetic inputs: reaction networks, initial states and run settings.

This module holds data only. It contains none of the simulation arithmetic, so
both the CPU oracle (in the tests) and the CUDA path can be fed from it.

A network is given the way the paper stores it (Sec. 5, "Implementations"):
sparse COO matrices of reactant coefficients sigma_jk and of net state change
v_k, plus one rate constant c_k per reaction (Eq. 1-2).  Reactions have at most
two reactant molecules, the limit the paper uses to keep the matrices in shared
memory (Sec. 5).

Generators:
  * ``lotka_volterra``     -- the predator-prey model of Table 4 (Sec. 5)
  * ``birth_death``        -- 0 -> A (k), A -> 0 (gamma)
  * ``dimerisation``       -- 2A -> B (c1), B -> 2A (c2)
  * ``isomerisation``      -- A -> B (k1), B -> A (k2)
  * ``random_mass_action`` -- random uni/bimolecular networks
  * ``poisson_x0``         -- Poisson initial counts
  * ``batched_networks``   -- thousands of random networks of uneven size

Rate constants of random networks are rounded to float32 after drawing so that
the same seed gives bit-identical inputs on x86-64 and aarch64 hosts (libm's
exp may differ in the last bit between the two).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Seed base for network generators: config index is added to it.
GEN_SEED_BASE = 20210301


@dataclasses.dataclass
class Network:
    """A mass-action reaction network in COO form.

    reac_rxn/reac_sp/reac_coef: reactant coefficient sigma_{sp,rxn} (> 0).
    stoi_rxn/stoi_sp/stoi_delta: net change v_k of species sp when rxn fires.
    c: rate constants, float64 [n_reactions].
    """

    n_species: int
    n_reactions: int
    reac_rxn: np.ndarray
    reac_sp: np.ndarray
    reac_coef: np.ndarray
    stoi_rxn: np.ndarray
    stoi_sp: np.ndarray
    stoi_delta: np.ndarray
    c: np.ndarray
    name: str = "network"

    def __post_init__(self):
        for f in ("reac_rxn", "reac_sp", "reac_coef", "stoi_rxn", "stoi_sp", "stoi_delta"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.int32))
        self.c = np.ascontiguousarray(self.c, dtype=np.float64)

    def with_rates(self, c) -> "Network":
        return dataclasses.replace(self, c=np.asarray(c, dtype=np.float64).copy())

    def dense_reactants(self) -> np.ndarray:
        """[M, N] reactant coefficient matrix (for small networks in tests)."""
        s = np.zeros((self.n_reactions, self.n_species), dtype=np.int64)
        np.add.at(s, (self.reac_rxn, self.reac_sp), self.reac_coef)
        return s

    def dense_stoich(self) -> np.ndarray:
        """[M, N] net state-change matrix v (row k = v_k)."""
        v = np.zeros((self.n_reactions, self.n_species), dtype=np.int64)
        np.add.at(v, (self.stoi_rxn, self.stoi_sp), self.stoi_delta)
        return v


def _from_lists(n_species: int, reactions: Sequence[Tuple[dict, dict, float]], name: str) -> Network:
    """Build a network from (reactants {sp: coef}, products {sp: coef}, c) triples."""
    rr, rs, rc, sr, ss, sd, cs = [], [], [], [], [], [], []
    for k, (reac, prod, c) in enumerate(reactions):
        for sp, coef in reac.items():
            rr.append(k); rs.append(sp); rc.append(coef)
        net = {}
        for sp, coef in reac.items():
            net[sp] = net.get(sp, 0) - coef
        for sp, coef in prod.items():
            net[sp] = net.get(sp, 0) + coef
        for sp, d in sorted(net.items()):
            if d != 0:
                sr.append(k); ss.append(sp); sd.append(d)
        cs.append(c)
    return Network(n_species, len(reactions), np.array(rr), np.array(rs), np.array(rc),
                   np.array(sr), np.array(ss), np.array(sd), np.array(cs, dtype=np.float64), name)


def lotka_volterra(c1: float = 10.0, c2: float = 0.01, c3: float = 10.0) -> Network:
    """Predator-prey model of Table 4: X -> 2X, X + Y -> 2Y, Y -> 0 (species X=0, Y=1)."""
    return _from_lists(2, [({0: 1}, {0: 2}, c1), ({0: 1, 1: 1}, {1: 2}, c2), ({1: 1}, {}, c3)],
                       "lotka_volterra")


def birth_death(k: float = 100.0, gamma: float = 1.0) -> Network:
    """0 -> A at rate k, A -> 0 at rate gamma*A."""
    return _from_lists(1, [({}, {0: 1}, k), ({0: 1}, {}, gamma)], "birth_death")


def dimerisation(c1: float = 0.001, c2: float = 0.1) -> Network:
    """2A -> B with propensity c1*A(A-1)/2, B -> 2A with c2*B (species A=0, B=1)."""
    return _from_lists(2, [({0: 2}, {1: 1}, c1), ({1: 1}, {0: 2}, c2)], "dimerisation")


def isomerisation(k1: float = 1.0, k2: float = 0.5) -> Network:
    """A -> B at k1*A, B -> A at k2*B (species A=0, B=1)."""
    return _from_lists(2, [({0: 1}, {1: 1}, k1), ({1: 1}, {0: 1}, k2)], "isomerisation")


def pure_birth(c: float = 1.0) -> Network:
    """0 -> A at constant rate c (the counting process is Poisson(c t))."""
    return _from_lists(1, [({}, {0: 1}, c)], "pure_birth")


def random_mass_action(n_species: int, n_reactions: int, seed: int, c_sigma: float = 1.0,
                       name: str = "random") -> Network:
    """Random uni/bimolecular mass-action network.

    Each reaction has order 1 or 2 with probability 1/2; reactant species are
    drawn uniformly with replacement (so 2A occurs); the product count is
    uniform in {0, 1, 2} with uniform species; v = products - reactants;
    c ~ lognormal(0, c_sigma), rounded to float32.
    """
    rng = np.random.default_rng(seed)
    M, N = int(n_reactions), int(n_species)
    order = rng.integers(1, 3, size=M)
    r0 = rng.integers(0, N, size=M)
    r1 = rng.integers(0, N, size=M)
    npro = rng.integers(0, 3, size=M)
    p0 = rng.integers(0, N, size=M)
    p1 = rng.integers(0, N, size=M)
    c = np.exp(c_sigma * rng.standard_normal(M)).astype(np.float32).astype(np.float64)

    k = np.arange(M)
    two = order == 2
    # reactant COO; 2A is stored as one entry with coefficient 2
    same = two & (r0 == r1)
    diff = two & (r0 != r1)
    reac_rxn = np.concatenate([k[~two], k[same], k[diff], k[diff]])
    reac_sp = np.concatenate([r0[~two], r0[same], r0[diff], r1[diff]])
    reac_coef = np.concatenate([np.ones((~two).sum()), np.full(same.sum(), 2),
                                np.ones(diff.sum()), np.ones(diff.sum())])
    # net change: -reactants + products, duplicates summed, zeros dropped
    rows = np.concatenate([k, k[two], k[npro >= 1], k[npro >= 2]])
    cols = np.concatenate([r0, r1[two], p0[npro >= 1], p1[npro >= 2]])
    vals = np.concatenate([-np.ones(M), -np.ones(two.sum()), np.ones((npro >= 1).sum()),
                           np.ones((npro >= 2).sum())])
    key = rows.astype(np.int64) * N + cols
    uk, inv = np.unique(key, return_inverse=True)
    sums = np.zeros(uk.shape[0], dtype=np.int64)
    np.add.at(sums, inv, vals.astype(np.int64))
    nz = sums != 0
    order_idx = np.argsort(reac_rxn, kind="stable")
    return Network(N, M, reac_rxn[order_idx], reac_sp[order_idx], reac_coef[order_idx],
                   (uk[nz] // N), (uk[nz] % N), sums[nz], c, name)


def poisson_x0(n_species: int, mean: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.poisson(mean, size=int(n_species)).astype(np.int32)


@dataclasses.dataclass
class BatchItem:
    net: Network
    x0: np.ndarray
    t_end: float


def batched_networks(n_nets: int = 4096, m_lo: int = 4, m_hi: int = 4096, seed: int = GEN_SEED_BASE + 4,
                     x0_mean: float = 50.0, t_lo: float = 1.0, t_hi: float = 10.0,
                     c_sigma: float = 1.0) -> List[BatchItem]:
    """Networks of uneven size: M ~ U{m_lo..m_hi}, N = max(1, M // 4), t_end ~ U[t_lo, t_hi]."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=n_nets)
    seeds = rng.integers(0, 2**31 - 1, size=n_nets)
    tends = np.round(rng.uniform(t_lo, t_hi, size=n_nets), 6)
    out = []
    for i in range(n_nets):
        M = int(ms[i])
        N = max(1, M // 4)
        net = random_mass_action(N, M, int(seeds[i]), c_sigma, name=f"batch{i}")
        out.append(BatchItem(net, poisson_x0(N, x0_mean, int(seeds[i]) + 1), float(tends[i])))
    return out


# --------------------------------------------------------------------------------------
# The five evaluation workloads at their benchmarked sizes.
# --------------------------------------------------------------------------------------

def lv_config(n_traj: int = 64):
    """Lotka-Volterra of Table 4 with c = (10, 0.01, 10), X0 = Y0 = 1000, t_end = 5, grid 0.01."""
    return dict(net=lotka_volterra(), x0=np.array([1000, 1000], np.int32), t_end=5.0,
                sample_dt=0.01, n_traj=n_traj, seed=1)


# Per-trajectory event cap of the ensemble workload.  A Lotka-Volterra trajectory
# whose predators die out lets the prey grow until int32 overflow (~2^31 events in
# one thread); trajectories to t = 10 fire at most ~3.1e5 events otherwise.  Capped
# trajectories end with status MAX_EVENTS and are reported, not dropped.
ENSEMBLE_MAX_EVENTS = 1_000_000


def ensemble_configs(n_traj: int = 1 << 20):
    """Lotka-Volterra, birth-death (k=100, gamma=1, A0=0) and dimerisation (0.001/0.1, A0=1000, B0=0),
    each n_traj trajectories to t_end = 10."""
    cap = ENSEMBLE_MAX_EVENTS
    return [
        dict(net=lotka_volterra(), x0=np.array([1000, 1000], np.int32), t_end=10.0, n_traj=n_traj, seed=1,
             max_events=cap),
        dict(net=birth_death(), x0=np.array([0], np.int32), t_end=10.0, n_traj=n_traj, seed=1, max_events=cap),
        dict(net=dimerisation(), x0=np.array([1000, 0], np.int32), t_end=10.0, n_traj=n_traj, seed=1,
             max_events=cap),
    ]


def large_network_config(n_species: int = 10_000, n_reactions: int = 1_000_000, n_traj: int = 16,
                         max_events: int = 1_000_000):
    """Random network, c ~ lognormal(0,1), X0 ~ Poisson(100), run for max_events events (t_end = inf)."""
    seed = GEN_SEED_BASE + 2
    net = random_mass_action(n_species, n_reactions, seed, 1.0, name="large")
    return dict(net=net, x0=poisson_x0(n_species, 100.0, seed + 1), t_end=float("inf"),
                max_events=max_events, n_traj=n_traj, seed=1)


def grad_config(n_traj: int = 65536):
    """Random network M=64, N=16, c ~ lognormal(0, 0.5), X0 ~ Poisson(200), t_end = 5."""
    seed = GEN_SEED_BASE + 4 + 1
    net = random_mass_action(16, 64, seed, 0.5, name="grad64")
    return dict(net=net, x0=poisson_x0(16, 200.0, seed + 1), t_end=5.0, n_traj=n_traj, seed=1)
