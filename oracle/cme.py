"""Exact transient law of tiny closed reaction systems (TEST INFRASTRUCTURE).

The Chemical Master Equation governs the probability of X(t) being in each
state (Methods section, stochastic formulation).  It is intractable for large
systems, but for a closed system with a handful of molecules the reachable
state space is finite, so P(t) = P(0) expm(Q t) with Q the CTMC generator.
This gives the exact distribution that sample paths of the SSA (and of
tau-leaping when every reaction is critical) must follow.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def _propensity(reactants, c, x):
    a = c
    for s, coef in reactants:
        if coef == 1:
            a *= x[s]
        elif coef == 2:
            a *= x[s] * (x[s] - 1) / 2.0
        else:
            raise ValueError("order > 2")
    return a


def reachable_states(network, x0, limit=20000):
    """Breadth-first enumeration of the states reachable from x0."""
    nu = network.stoichiometry().T  # [M, N]
    start = tuple(int(v) for v in x0)
    index = {start: 0}
    order = [start]
    q = 0
    while q < len(order):
        x = order[q]
        q += 1
        for j, row in enumerate(network.reactants):
            if _propensity(row, 1.0, x) <= 0:
                continue
            y = tuple(int(a + b) for a, b in zip(x, nu[j]))
            if min(y) < 0:
                continue
            if y not in index:
                if len(order) >= limit:
                    raise ValueError("state space too large for the exact CME")
                index[y] = len(order)
                order.append(y)
    return order, index


def transient_distribution(network, rates, x0, times):
    """P(X(t) = state) for each t in ``times``.

    Returns (states [K, N] int, probs [len(times), K]).
    """
    states, index = reachable_states(network, x0)
    K = len(states)
    nu = network.stoichiometry().T
    Q = np.zeros((K, K))
    for a_idx, x in enumerate(states):
        for j, row in enumerate(network.reactants):
            a = _propensity(row, float(rates[j]), x)
            if a <= 0:
                continue
            y = tuple(int(p + d) for p, d in zip(x, nu[j]))
            b_idx = index[y]
            Q[a_idx, b_idx] += a
            Q[a_idx, a_idx] -= a
    p0 = np.zeros(K)
    p0[0] = 1.0
    out = []
    for t in times:
        out.append(p0 @ scipy.linalg.expm(Q * float(t)))
    probs = np.clip(np.asarray(out), 0.0, None)
    return np.asarray(states, dtype=np.int64), probs
