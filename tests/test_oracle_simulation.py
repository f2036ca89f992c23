"""Pins for the oracle's simulation loop (exact SSA and tau-leaping).

Checked against: closed-form laws (birth-death Poisson, isomerization
binomial, pure production Poisson), the exact Chemical Master Equation of
tiny closed systems (matrix exponential of the generator), the exact mean of
the explicit tau-leap recursion, hand-derived tau' values for one-reaction
networks, the mean-field ODE limit, and invariants (conservation laws,
non-negativity, status semantics)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import cme, rre
from conftest import chi2_pvalue
from paper_1309_7695_b300 import inputs

SSA = oracle.MODE_EXACT_SSA
TAU = oracle.MODE_TAU_LEAP


def run(net, rates, x0, reps, t_end, times, mode, seed=0, **kw):
    b = inputs.replicate_batch(net, rates, x0, reps, t_end, 2)
    b.sample_times = np.asarray(times, dtype=np.float64)
    return oracle.simulate(net, b.params, b.x0, t_end, b.sample_times, seed=seed,
                           opts=oracle.default_opts(mode=mode, **kw))


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("mode", [SSA, TAU])
def test_birth_death_poisson_law(mode):
    # 0 -> X (k = 10), X -> 0 (g = 0.1), X(0) = 0: X(t) ~ Poisson(100 (1 - e^{-0.1 t})).
    # Counts stay near 100, where tau-leaping falls back to exact SSA steps.
    times = [2.0, 5.0, 10.0, 30.0]
    s, st = run(inputs.birth_death(), [10.0, 0.1], [0], 20_000, 30.0, times, mode, seed=1)
    assert np.all(st["status"] == 0)
    for q, t in enumerate(times):
        lam = 100.0 * (1.0 - math.exp(-0.1 * t))
        x = s[:, q, 0]
        sup = np.arange(x.max() + 1)
        pr = stats.poisson.pmf(sup, lam)
        pr[-1] += stats.poisson.sf(x.max(), lam)
        assert chi2_pvalue(np.bincount(x, minlength=len(sup)), pr) > 1e-3, t


def test_isomerization_binomial_law():
    # A -> B (k = 1), A(0) = 100: A(t) ~ Binomial(100, e^{-t}); B = 100 - A.
    times = [0.0, 0.5, 1.0, 2.0]
    s, _ = run(inputs.isomerization(), [1.0], [100, 0], 20_000, 2.0, times, SSA, seed=2)
    assert np.all(s[:, :, 0] + s[:, :, 1] == 100)
    assert np.all(s[:, 0, 0] == 100)
    for q, t in enumerate(times[1:], start=1):
        a = s[:, q, 0]
        sup = np.arange(101)
        pr = stats.binom.pmf(sup, 100, math.exp(-t))
        assert chi2_pvalue(np.bincount(a, minlength=101), pr) > 1e-3, t


def test_pure_production_is_one_exact_leap_per_interval():
    # A -> A + B: nu_A = 0 so it is never critical and A bounds nothing; B is
    # no reactant, so tau' is infinite and every leap runs to the next sample
    # time.  B(t) ~ Poisson(c A t) exactly.
    net = inputs.Network(2, [[(0, 1)]], [[(0, 1), (1, 1)]])
    times = [0.0, 1.0, 2.5, 4.0]
    s, st = run(net, [0.7], [20, 0], 20_000, 4.0, times, TAU, seed=3)
    assert np.all(st["leaps"] == 3) and np.all(st["ssa_steps"] == 0)
    for q, t in enumerate(times):
        b = s[:, q, 1]
        lam = 0.7 * 20 * t
        if lam == 0:
            assert np.all(b == 0)
            continue
        sup = np.arange(b.max() + 1)
        pr = stats.poisson.pmf(sup, lam)
        pr[-1] += stats.poisson.sf(b.max(), lam)
        assert chi2_pvalue(np.bincount(b, minlength=len(sup)), pr) > 1e-3


# ------------------------------------------------- exact CME, tiny systems

TINY_CASES = [
    ("michaelis_menten", inputs.michaelis_menten(), [1.0, 0.5, 0.7], [2, 3, 0, 0]),
    ("dimerization", inputs.dimerization(), [0.2, 0.5], [8, 0]),
]


@pytest.mark.parametrize("name,net,rates,x0", TINY_CASES, ids=[c[0] for c in TINY_CASES])
@pytest.mark.parametrize("mode", [SSA, TAU])
def test_tiny_system_matches_exact_cme(name, net, rates, x0, mode):
    # With every count below n_c = 10 each reaction that can fire is critical,
    # tau' is infinite and tau-leaping fires one reaction per step at the
    # exponential time tau'' -- the same law as the exact SSA.
    times = [0.3, 1.0, 3.0]
    states, probs = cme.transient_distribution(net, rates, x0, times)
    s, st = run(net, rates, x0, 40_000, 3.0, times, mode, seed=4)
    if mode == TAU:
        assert st["ssa_steps"].sum() == 0 and st["leaps"].sum() > 0
    lookup = {tuple(v): i for i, v in enumerate(states)}
    for q in range(len(times)):
        idx = np.array([lookup[tuple(v)] for v in s[:, q, :]])
        counts = np.bincount(idx, minlength=len(states))
        assert chi2_pvalue(counts, probs[q]) > 1e-3, (name, times[q])


# ------------------------------------------- tau-leap at large counts

@pytest.mark.parametrize("eps", [0.03, 0.01, 0.003])
def test_isomerization_tau_leap_mean_follows_leap_recursion(eps):
    # A -> B with k = 1, A(0) = 1e4.  tau' = min(eps/k, eps^2 A/k) (g_A = 1,
    # mu = -kA, sigma^2 = kA) equals eps/k while A >= 1/eps, which holds here
    # throughout (A stays above 3000); the reaction is noncritical and
    # A_{n+1} = A_n - Poisson(k A_n tau), so E[A_n] = A0 (1 - eps)^n and
    # Var[A_{n+1}] = (1 - eps)^2 Var[A_n] + eps E[A_n].  Sample times are
    # multiples of 0.3, an integer number of steps of eps.  At eps = 0.003
    # the SSA-fallback threshold 10/a0 <= 2.5e-3 stays below tau'.
    times = [0.0, 0.3, 0.6, 0.9]
    reps = 4000
    s, st = run(inputs.isomerization(), [1.0], [10_000, 0], reps, 0.9, times, TAU, seed=5,
                eps=eps)
    assert np.all(st["ssa_steps"] == 0)
    steps_per_interval = round(0.3 / eps)
    mean, var = 10_000.0, 0.0
    for q in range(1, len(times)):
        for _ in range(steps_per_interval):
            var = (1 - eps) ** 2 * var + eps * mean
            mean = mean * (1 - eps)
        got = s[:, q, 0].astype(np.float64)
        se = math.sqrt(var / reps)
        assert abs(got.mean() - mean) < 5 * se, (q, got.mean(), mean)
        exact_ssa_mean = 10_000.0 * math.exp(-times[q])
        # the leap bias relative to the exact process is O(eps)
        assert abs(mean - exact_ssa_mean) / exact_ssa_mean < 0.75 * eps * times[q] + 1e-9


def test_tau_prime_one_reaction_closed_forms():
    eps = 0.03
    o = oracle.default_opts(eps=eps)
    iso = inputs.isomerization()
    # A -> B, x_A = 10000: tau' = min(eps x/(k x), (eps x)^2/(k x)) = eps/k
    q = oracle.leap_quantities(iso, [2.0], [10_000, 5], o)
    assert q["tau1"] == pytest.approx(eps / 2.0, rel=1e-15)
    assert not q["crit"][0] and q["a0c"] == 0.0
    # x_A = 20: eps x < 1 so the bound is 1: tau' = min(1/(k x), 1/(k x))
    q = oracle.leap_quantities(iso, [2.0], [20, 0], o)
    assert q["tau1"] == pytest.approx(1.0 / 40.0, rel=1e-15)
    # x_A = 9 < n_c: critical, no noncritical reaction -> tau' infinite
    q = oracle.leap_quantities(iso, [2.0], [9, 0], o)
    assert q["crit"][0] and math.isinf(q["tau1"]) and q["a0c"] == q["a0"] == 18.0
    # 2A -> B only: g = 2 + 1/(x-1); mu = -2a, sigma^2 = 4a, a = c x(x-1)/2
    dim = inputs.Network(2, [[(0, 2)]], [[(1, 1)]])
    x = 1000
    a = 0.01 * x * (x - 1) / 2
    g = 2.0 + 1.0 / (x - 1)
    bound = max(eps * x / g, 1.0)
    q = oracle.leap_quantities(dim, [0.01], [x, 0], o)
    assert q["a"][0] == pytest.approx(a, rel=1e-15)
    assert q["tau1"] == pytest.approx(min(bound / (2 * a), bound ** 2 / (4 * a)), rel=1e-14)
    # A + B -> C: g = 2 for both; species with the smaller count binds
    abc = inputs.Network(3, [[(0, 1), (1, 1)]], [[(2, 1)]])
    xa, xb, c = 400, 3000, 1e-3
    a = c * xa * xb
    cand = [max(eps * v / 2.0, 1.0) for v in (xa, xb)]
    expect = min(min(bnd / a, bnd ** 2 / a) for bnd in cand)
    q = oracle.leap_quantities(abc, [c], [xa, xb, 0], o)
    assert q["tau1"] == pytest.approx(expect, rel=1e-14)
    # a species that is only a product of noncritical reactions bounds nothing
    q = oracle.leap_quantities(abc, [c], [xa, xb, 10**6], o)
    assert q["tau1"] == pytest.approx(expect, rel=1e-14)
    # the same with the counts swapped: now the second reactant binds, so it
    # must be a member of I_rs as well
    q = oracle.leap_quantities(abc, [c], [xb, xa, 0], o)
    assert q["tau1"] == pytest.approx(expect, rel=1e-14)
    # birth-death at X = 0: the death reaction has a = 0 but is not critical,
    # so X is a reactant species of a noncritical reaction and bounds the
    # step through the birth flux: tau' = min(1/k, 1/k) with bound 1.
    q = oracle.leap_quantities(inputs.birth_death(), [10.0, 0.1], [0], o)
    assert q["tau1"] == pytest.approx(0.1, rel=1e-15) and not q["crit"].any()


def test_critical_set_uses_net_change():
    # 2A -> A (nu_A = -1, L = x_A) versus 2A -> B (nu_A = -2, L = floor(x_A/2)).
    o = oracle.default_opts()
    net = inputs.Network(2, [[(0, 2)], [(0, 2)]], [[(0, 1)], [(1, 1)]])
    q = oracle.leap_quantities(net, [1.0, 1.0], [15, 0], o)
    assert list(q["crit"]) == [False, True]      # L = 15 and 7
    q = oracle.leap_quantities(net, [1.0, 1.0], [25, 0], o)
    assert list(q["crit"]) == [False, False]     # L = 25 and 12
    q = oracle.leap_quantities(net, [1.0, 1.0], [1, 0], o)
    assert list(q["crit"]) == [False, False]     # a_j = 0: never critical
    assert q["a0"] == 0.0
    # the threshold itself (CGP 2005): critical iff L < n_c, so L = n_c is not
    q = oracle.leap_quantities(net, [1.0, 1.0], [20, 0], o)
    assert list(q["crit"]) == [False, False]     # L = 20 and 10
    q = oracle.leap_quantities(net, [1.0, 1.0], [19, 0], o)
    assert list(q["crit"]) == [False, True]      # L = 19 and 9
    iso = inputs.isomerization()
    assert not oracle.leap_quantities(iso, [1.0], [10, 0], o)["crit"][0]
    assert oracle.leap_quantities(iso, [1.0], [9, 0], o)["crit"][0]
    q = oracle.leap_quantities(iso, [1.0], [9, 0], oracle.default_opts(n_c=9))
    assert not q["crit"][0]


def test_critical_reactions_fire_at_their_exact_rate_beside_leaps():
    # A -> 0 with A(0) = 8 < n_c is critical throughout, beside B -> 0 with
    # B(0) = 1e5, which leaps.  tau'' is redrawn from the critical total a0c at
    # every step and, being exponential, is memoryless, so the critical firings
    # form the exact SSA of A alone: A(t) ~ Binomial(8, e^{-t}) at every t,
    # however many leaps of B happen meanwhile.
    net = inputs.Network(2, [[(0, 1)], [(1, 1)]], [[], []])
    times = [0.25, 0.5, 1.0, 2.0]
    reps = 20_000
    s, st = run(net, [1.0, 1.0], [8, 100_000], reps, 2.0, times, TAU, seed=9)
    assert np.all(st["status"] == 0)
    assert st["leaps"].mean() > 50          # B does leap
    for q, t in enumerate(times):
        counts = np.bincount(s[:, q, 0], minlength=9)
        probs = stats.binom.pmf(np.arange(9), 8, math.exp(-t))
        assert chi2_pvalue(counts, probs) > 1e-3, t


def test_mean_field_limit():
    # Kurtz (Methods): as counts scale by Omega (bimolecular constants by
    # 1/Omega) the stochastic mean approaches the reaction-rate equations.
    # (a) small Omega, dimerization 2A <-> B: the oracle's mean equals the
    #     exact CME mean within sampling error, and that mean sits a clear
    #     O(1/Omega) distance from the ODE;
    net = inputs.dimerization()
    times = np.array([0.5, 2.0, 5.0])
    gaps = {}
    for omega, reps in ((1, 20000), (4, 8000)):
        rates, x0 = [0.1 / omega, 0.5], [20 * omega, 0]
        ode = rre.integrate(net, rates, np.array(x0), np.concatenate([[0.0], times]))[1:, 0]
        states, probs = cme.transient_distribution(net, rates, x0, times)
        exact_mean = probs @ states[:, 0]
        s, _ = run(net, rates, x0, reps, 5.0, times, TAU, seed=6, eps=0.01)
        a = s[:, :, 0].astype(np.float64)
        se = a.std(axis=0) / math.sqrt(reps)
        assert np.all(np.abs(a.mean(axis=0) - exact_mean) < 4 * se)
        gaps[omega] = np.abs(exact_mean - ode) / (20 * omega)
    assert np.all(gaps[1] > 3e-3)
    np.testing.assert_allclose(gaps[1] / gaps[4], 4.0, rtol=0.25)
    # (b) large counts, Michaelis-Menten at Omega = 100 with real leaps: the
    #     tau-leap mean is within 0.5% of the ODE solution.
    mm = inputs.michaelis_menten()
    omega = 100
    rates = [0.005 / omega, 0.1, 0.1]
    x0 = [200 * omega, 500 * omega, 0, 0]
    t = np.array([0.0, 1.0, 2.0, 5.0])
    ode = rre.integrate(mm, rates, x0, t)
    s, st = run(mm, rates, x0, 200, 5.0, t, TAU, seed=6, eps=0.01)
    assert np.all(st["status"] == 0) and st["leaps"].min() > 100
    assert np.abs(s.mean(axis=0) - ode).max() / (500 * omega) < 5e-3


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("mode", [SSA, TAU])
def test_mm_sweep_conservation_and_first_sample(mode):
    b = inputs.mm_batch(256, seed=3)
    s, st = oracle.simulate_batch(b, seed=9, opts=oracle.default_opts(mode=mode))
    assert np.all(st["status"] == 0)
    assert np.all(s[:, :, 0] + s[:, :, 2] == 200)
    assert np.all(s[:, :, 1] + s[:, :, 2] + s[:, :, 3] == 500)
    assert np.all(s[:, 0, :] == b.x0)
    assert np.all(st["t_final"] == b.t_end)
    assert np.all(st["firings"] == st["ssa_steps"] + (st["firings"] - st["ssa_steps"]))


def test_random_network_nonnegative_and_subset_reproducible():
    b = inputs.random_batch(16, 32, 64, seed=2, t_end=5.0, n_samples=6)
    o = oracle.default_opts(max_attempts=200_000)
    s, st = oracle.simulate_batch(b, seed=4, opts=o)
    assert s.min() >= 0
    assert np.all(s[:, 0, :] == b.x0)
    rows = [5, 17, 63]
    s2, st2 = oracle.simulate_batch(b, seed=4, opts=o, rows=rows)
    assert np.array_equal(s2, s[rows])
    assert np.array_equal(st2, st[rows])
    s3, _ = oracle.simulate_batch(b, seed=5, opts=o)
    assert not np.array_equal(s3, s)


def test_frozen_system_and_empty_inputs():
    iso = inputs.isomerization()
    s, st = run(iso, [1.0], [0, 7], 3, 10.0, [0.0, 5.0, 10.0], TAU)
    assert np.all(s == np.array([0, 7])) and np.all(st["status"] == 0)
    assert np.all(st["t_final"] == 10.0) and np.all(st["attempts"] == 0)
    s, st = run(iso, [1.0], [5, 0], 2, 0.0, [0.0], TAU)
    assert np.all(s[:, 0] == [5, 0]) and np.all(st["attempts"] == 0)
    s, st = run(iso, [1.0], [5, 0], 0, 1.0, [0.0, 1.0], TAU)
    assert s.shape == (0, 2, 2)


def test_step_limit_keeps_last_state():
    b = inputs.random_batch(8, 16, 4, seed=1, t_end=50.0, n_samples=11)
    s, st = oracle.simulate_batch(b, opts=oracle.default_opts(max_attempts=5))
    for r in range(4):
        if st["status"][r] == 1:
            assert st["attempts"][r] == 5
            last = s[r, -1]
            assert np.all(s[r, np.searchsorted(b.sample_times, st["t_final"][r], "right"):] == last)


def test_explosion_reports_overflow():
    # A -> 2A with c = 1 grows like e^t: counts pass 2^31 - 1 before t = 100
    net = inputs.Network(1, [[(0, 1)]], [[(0, 2)]])
    s, st = run(net, [1.0], [1000], 4, 100.0, np.linspace(0, 100, 11), TAU)
    assert np.all(st["status"] == 2)
    assert s.max() <= 2**31 - 1
    assert np.all(s[:, -1, 0] == s[:, -2, 0])
