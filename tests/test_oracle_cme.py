"""Pins of the exact CME solver (oracle/cme.py) against closed forms.

The solver is the reference law for the tiny-system tests of the oracle and
of fast mode, so it is checked here on systems whose transient law is known
in closed form, independently of any simulation:
  - isomerization A -> B from A0: A(t) ~ Binomial(A0, e^{-ct});
  - reversible isomerization A <-> B from (A0, 0): every molecule is an
    independent two-state chain, so A(t) ~ Binomial(A0, p(t)) with
    p(t) = c2/(c1+c2) + c1/(c1+c2) e^{-(c1+c2)t} (unequal rates catch a
    transposed generator);
  - dimerization 2A -> B from A0 = 3: the only event has propensity
    c * 3*2/2 = 3c, so P(A = 3) = e^{-3ct} (catches x^2/2 or x(x-1) in place
    of the combinatorial x(x-1)/2);
  - A + B -> C from (2, 3): a pure-birth chain with rates 6c then 2c, so
    P(one event by t) = 6/(6-2) (e^{-2ct} - e^{-6ct}) and P(two) is the rest.
Each law is compared state by state within 1e-10."""
import math

import numpy as np
from scipy import stats

from oracle import cme
from paper_1309_7695_b300 import inputs


def _law_of_species(states, probs, species):
    """Marginal law of one species: {count: probability} per time."""
    out = []
    for row in probs:
        d = {}
        for s, p in zip(states, row):
            d[int(s[species])] = d.get(int(s[species]), 0.0) + float(p)
        out.append(d)
    return out


def test_isomerization_is_binomial():
    A0, c, times = 30, 0.7, [0.1, 1.0, 3.0]
    states, probs = cme.transient_distribution(inputs.isomerization(), [c], [A0, 0], times)
    assert np.all(states.sum(axis=1) == A0)
    for t, law in zip(times, _law_of_species(states, probs, 0)):
        want = stats.binom.pmf(np.arange(A0 + 1), A0, math.exp(-c * t))
        got = np.array([law.get(a, 0.0) for a in range(A0 + 1)])
        assert np.max(np.abs(got - want)) < 1e-10, t


def test_reversible_isomerization_is_binomial():
    A0, c1, c2, times = 20, 1.3, 0.4, [0.05, 0.5, 2.0, 8.0]
    net = inputs.Network(2, [[(0, 1)], [(1, 1)]], [[(1, 1)], [(0, 1)]], name="A<->B")
    states, probs = cme.transient_distribution(net, [c1, c2], [A0, 0], times)
    for t, law in zip(times, _law_of_species(states, probs, 0)):
        p = c2 / (c1 + c2) + c1 / (c1 + c2) * math.exp(-(c1 + c2) * t)
        want = stats.binom.pmf(np.arange(A0 + 1), A0, p)
        got = np.array([law.get(a, 0.0) for a in range(A0 + 1)])
        assert np.max(np.abs(got - want)) < 1e-10, t


def test_dimerization_uses_combinatorial_propensity():
    c, times = 0.9, [0.2, 1.0, 2.5]
    net = inputs.Network(2, [[(0, 2)]], [[(1, 1)]], name="2A->B")
    states, probs = cme.transient_distribution(net, [c], [3, 0], times)
    for t, law in zip(times, _law_of_species(states, probs, 0)):
        assert abs(law[3] - math.exp(-3 * c * t)) < 1e-10
        assert abs(law[1] - (1 - math.exp(-3 * c * t))) < 1e-10
        assert set(law) == {1, 3}


def test_bimolecular_pure_birth_chain():
    c, times = 0.35, [0.1, 0.7, 3.0]
    net = inputs.Network(3, [[(0, 1), (1, 1)]], [[(2, 1)]], name="A+B->C")
    states, probs = cme.transient_distribution(net, [c], [2, 3, 0], times)
    for t, law in zip(times, _law_of_species(states, probs, 2)):
        p0 = math.exp(-6 * c * t)
        p1 = 6 / (6 - 2) * (math.exp(-2 * c * t) - math.exp(-6 * c * t))
        assert abs(law[0] - p0) < 1e-10
        assert abs(law[1] - p1) < 1e-10
        assert abs(law[2] - (1 - p0 - p1)) < 1e-10
