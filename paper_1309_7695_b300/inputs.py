"""Seeded synthetic inputs: reaction networks, parameter sweeps, initial counts.

This module only *generates inputs*.  It holds none of the simulation
method's arithmetic (no propensities, no tau selection, no random streams of
the method), so both the CPU oracle and the CUDA engine can consume what it
produces without sharing any implementation.

A network is a set of mass-action reactions over ``n_species`` species
(Methods section: a reaction set acting on the state vector X(t) of molecule
counts).  Each reaction j has a reactant multiset and a product multiset, both
given as ``(species, coefficient)`` pairs.  Reaction order (the sum of
reactant coefficients) is at most 2.

Parameterizations follow the paper's motivation (Aims and motivation: many
simulations of one model, each with its own kinetic constants and initial
molecular amounts): ``params[s, j]`` is the stochastic rate constant c_j of
simulation s and ``x0[s, i]`` its initial count of species i.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    """A mass-action reaction network (species count + reactions)."""

    n_species: int
    reactants: list  # per reaction: list of (species, coef)
    products: list  # per reaction: list of (species, coef)
    name: str = "network"
    species_names: list = field(default_factory=list)

    @property
    def n_reactions(self) -> int:
        """Number of reactions M."""
        return len(self.reactants)

    def csr(self) -> dict:
        """Reactant and product lists as int32 CSR arrays.

        Entries of each row are sorted by species index; a species appears at
        most once per row (its coefficient carries the multiplicity).
        """
        out = {}
        for side, rows in (("react", self.reactants), ("prod", self.products)):
            ptr = [0]
            sp, cf = [], []
            for row in rows:
                merged = {}
                for s, c in row:
                    merged[int(s)] = merged.get(int(s), 0) + int(c)
                for s in sorted(merged):
                    sp.append(s)
                    cf.append(merged[s])
                ptr.append(len(sp))
            out[f"{side}_ptr"] = np.asarray(ptr, dtype=np.int32)
            out[f"{side}_species"] = np.asarray(sp, dtype=np.int32)
            out[f"{side}_coef"] = np.asarray(cf, dtype=np.int32)
        return out

    def stoichiometry(self) -> np.ndarray:
        """Dense net-change matrix nu[i, j] = products - reactants (int64)."""
        nu = np.zeros((self.n_species, self.n_reactions), dtype=np.int64)
        for j, row in enumerate(self.reactants):
            for s, c in row:
                nu[s, j] -= c
        for j, row in enumerate(self.products):
            for s, c in row:
                nu[s, j] += c
        return nu

    def orders(self) -> np.ndarray:
        """Reaction orders (sum of reactant coefficients), int32 [M]."""
        return np.asarray([sum(c for _, c in row) for row in self.reactants], dtype=np.int32)


@dataclass
class Batch:
    """One sweep: a network plus per-simulation constants and initial counts."""

    network: Network
    params: np.ndarray  # float64 [n_sims, M]
    x0: np.ndarray  # int32 [n_sims, N]
    t_end: float
    sample_times: np.ndarray  # float64 [S], ascending, within [0, t_end]

    @property
    def n_sims(self) -> int:
        """Number of simulations (parameter rows)."""
        return int(self.params.shape[0])


# ---------------------------------------------------------------- networks

def michaelis_menten() -> Network:
    """E + S -> ES (k1), ES -> E + S (k2), ES -> E + P (k3); species E,S,ES,P."""
    return Network(
        n_species=4,
        reactants=[[(0, 1), (1, 1)], [(2, 1)], [(2, 1)]],
        products=[[(2, 1)], [(0, 1), (1, 1)], [(0, 1), (3, 1)]],
        name="michaelis_menten",
        species_names=["E", "S", "ES", "P"],
    )


def birth_death() -> Network:
    """0 -> X (rate k), X -> 0 (rate g)."""
    return Network(1, [[], [(0, 1)]], [[(0, 1)], []], name="birth_death", species_names=["X"])


def isomerization() -> Network:
    """A -> B (rate k)."""
    return Network(2, [[(0, 1)]], [[(1, 1)]], name="isomerization", species_names=["A", "B"])


def dimerization() -> Network:
    """2A -> B (c1), B -> 2A (c2): exercises the 2X propensity and its g_i rule."""
    return Network(2, [[(0, 2)], [(1, 1)]], [[(1, 1)], [(0, 2)]], name="dimerization",
                   species_names=["A", "B"])


def random_network(n_species: int, n_reactions: int, seed: int) -> Network:
    """Random mass-action network with reaction orders 0/1/2 in ratio 1:2:1.

    Exactly floor(M/4) order-0, the order-2 count floor(M/4), and the rest
    order-1 reactions, in shuffled order.  Order 1: one reactant species drawn
    uniformly.  Order 2: two species drawn uniformly with replacement (a
    repeat gives 2X).  Products: a number of distinct species drawn uniformly
    from {0,1,2} (order >= 1) or {1,2} (order 0), each species uniform and
    each coefficient uniform in {1,2}.
    """
    rng = np.random.default_rng(np.random.PCG64([seed, n_species, n_reactions, 0x6E6574]))
    n0 = n_reactions // 4
    n2 = n_reactions // 4
    n1 = n_reactions - n0 - n2
    order = np.array([0] * n0 + [1] * n1 + [2] * n2)
    rng.shuffle(order)
    reactants, products = [], []
    for o in order:
        if o == 0:
            r = []
            n_prod = int(rng.integers(1, 3))
        elif o == 1:
            r = [(int(rng.integers(n_species)), 1)]
            n_prod = int(rng.integers(0, 3))
        else:
            a, b = (int(v) for v in rng.integers(n_species, size=2))
            r = [(a, 2)] if a == b else sorted([(a, 1), (b, 1)])
            n_prod = int(rng.integers(0, 3))
        n_prod = min(n_prod, n_species)
        sp = rng.choice(n_species, size=n_prod, replace=False) if n_prod else []
        p = sorted((int(s), int(rng.integers(1, 3))) for s in sp)
        reactants.append(r)
        products.append(p)
    return Network(n_species, reactants, products, name=f"random_{n_species}x{n_reactions}_s{seed}")


# ------------------------------------------------------------ sweep inputs

def log_uniform(rng: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    """Samples whose logarithm is uniform on [ln lo, ln hi]."""
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def uniform_sample_times(t_end: float, n_samples: int) -> np.ndarray:
    """s_k = k * t_end / (S - 1), k = 0..S-1 (the last one equals t_end)."""
    if n_samples == 1:
        return np.asarray([t_end], dtype=np.float64)
    k = np.arange(n_samples, dtype=np.float64)
    T = (k * t_end) / float(n_samples - 1)
    T[-1] = t_end          # (S-1) t_end / (S-1) can round one ulp above t_end
    return np.minimum(T, t_end)


def mm_batch(n_sims: int = 1024, seed: int = 0, t_end: float = 10.0, n_samples: int = 11,
             scale: float = 1.0) -> Batch:
    """Michaelis-Menten sweep: E,S,ES,P = 200,500,0,0; k1 ~ logU[1e-3,1e-2],
    k2,k3 ~ logU[1e-2,1].  ``scale`` multiplies the initial counts and divides
    k1 (the volume scaling used for the mean-field limit check)."""
    rng = np.random.default_rng(np.random.PCG64([seed, 0x6D6D]))
    k1 = log_uniform(rng, 1e-3, 1e-2, n_sims) / scale
    k2 = log_uniform(rng, 1e-2, 1.0, n_sims)
    k3 = log_uniform(rng, 1e-2, 1.0, n_sims)
    params = np.stack([k1, k2, k3], axis=1).astype(np.float64)
    x0 = np.tile(np.round(np.array([200, 500, 0, 0]) * scale).astype(np.int32), (n_sims, 1))
    return Batch(michaelis_menten(), params, x0, t_end, uniform_sample_times(t_end, n_samples))


def replicate_batch(network: Network, rates, x0, n_sims: int, t_end: float, n_samples: int) -> Batch:
    """``n_sims`` replicates of one parameterization (identical rows)."""
    params = np.tile(np.asarray(rates, dtype=np.float64), (n_sims, 1))
    x = np.tile(np.asarray(x0, dtype=np.int32), (n_sims, 1))
    return Batch(network, params, x, t_end, uniform_sample_times(t_end, n_samples))


def random_batch(n_species: int, n_reactions: int, n_sims: int, seed: int = 0,
                 x0_max: int = 1000, rate_lo: float = 1e-4, rate_hi: float = 1.0,
                 t_end: float = 100.0, n_samples: int = 101, network_seed: int | None = None) -> Batch:
    """Random-network sweep: rates ~ logU[rate_lo, rate_hi], x0 ~ U{0..x0_max}."""
    net = random_network(n_species, n_reactions, seed if network_seed is None else network_seed)
    rng = np.random.default_rng(np.random.PCG64([seed, n_species, n_reactions, 0x707261]))
    params = log_uniform(rng, rate_lo, rate_hi, (n_sims, n_reactions)).astype(np.float64)
    x0 = rng.integers(0, x0_max + 1, size=(n_sims, n_species)).astype(np.int32)
    return Batch(net, params, x0, t_end, uniform_sample_times(t_end, n_samples))


def hetero_groups(total_sims: int = 200_000, seed: int = 0,
                  reaction_counts=(8, 16, 32, 64, 128, 256, 384, 512)) -> list:
    """Heterogeneous persistent-batch workload: groups of (network, sweep).

    Groups are drawn until ``total_sims`` simulations exist: the network is
    uniform among the given sizes (species = reactions / 2), replicates
    ~ logU-int[16, 8192], t_end ~ logU[10, 1000], 101 sample times; the last
    group is truncated.  Returns a list of ``Batch`` objects.
    """
    rng = np.random.default_rng(np.random.PCG64([seed, 0x686574]))
    nets = [random_network(m // 2, m, seed + 17 * m) for m in reaction_counts]
    groups, done = [], 0
    while done < total_sims:
        idx = int(rng.integers(len(nets)))
        reps = int(np.floor(log_uniform(rng, 16, 8193, 1)[0]))
        reps = min(reps, total_sims - done)
        t_end = float(log_uniform(rng, 10.0, 1000.0, 1)[0])
        net = nets[idx]
        rates = log_uniform(rng, 1e-4, 1.0, net.n_reactions)
        x0 = rng.integers(0, 1001, size=net.n_species)
        groups.append(replicate_batch(net, rates, x0, reps, t_end, 101))
        done += reps
    return groups
