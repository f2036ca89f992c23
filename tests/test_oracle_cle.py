"""The Langevin (CLE) mode of the oracle: normal increments for leap means
>= 1000 against the normal law, a pure-production network where each
sample interval is exactly one such increment, agreement with Poisson leaps
in mean and variance at large counts, and identity with plain tau-leaping
when no leap mean reaches the threshold."""
import numpy as np
from scipy import stats

from paper_1309_7695_b300 import inputs


def test_normal_increments_have_the_poisson_moments(oracle_lib):
    for lam in (1000.0, 3.7e4, 1e6):
        k = oracle_lib.normal_leap_array(lam, 200_000, seed=7)
        n = len(k)
        assert abs(k.mean() - lam) < 4 * np.sqrt(lam / n)
        assert abs(k.var() / lam - 1.0) < 4 * np.sqrt(2.0 / n)
        assert k.min() >= 0
    z = (oracle_lib.normal_leap_array(1e6, 100_000, seed=8) - 1e6) / 1e3
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_cle_pure_production_is_one_normal_increment_per_interval(oracle_lib):
    # A -> A + B with c A >= 1000 per unit time: tau' is infinite (B is no
    # reactant, nu_A = 0), so each sample interval is one leap whose mean c A dt
    # is at or above the threshold: B(t) is a sum of rounded normal increments
    # with mean c A t and variance c A t (plus 1/12 per increment from rounding).
    net = inputs.Network(2, [[(0, 1)]], [[(0, 1), (1, 1)]])
    T = np.array([0.0, 1.0, 2.5, 4.0])
    n = 20_000
    s, st = oracle_lib.simulate(net, np.full((n, 1), 1.0), np.tile([1000, 0], (n, 1)).astype(np.int32), 4.0, T,
                                seed=3, opts=oracle_lib.default_opts(mode=oracle_lib.MODE_CLE))
    assert np.all(st["leaps"] == 3) and np.all(st["ssa_steps"] == 0)
    for c in range(1, len(T)):
        m = 1000.0 * T[c]
        b = s[:, c, 1].astype(np.float64)
        assert abs(b.mean() - m) < 4 * np.sqrt(m / n)
        assert abs(b.var() - (m + c / 12.0)) < 4 * m * np.sqrt(2.0 / n)
    z = (s[:, 1, 1] - 1000.0) / np.sqrt(1000.0)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_cle_birth_death_matches_poisson_leaps_in_mean_and_variance(oracle_lib):
    # the Langevin increment has the mean and variance of the Poisson count it
    # replaces, so at large counts the two leap schemes agree in both moments
    net = inputs.birth_death()
    k, g, n = 2e5, 1.0, 4000
    T = np.array([0.0, 0.5, 2.0, 5.0])
    params = np.tile([k, g], (n, 1))
    x0 = np.zeros((n, 1), dtype=np.int32)
    runs = [oracle_lib.simulate(net, params, x0, 5.0, T, seed=sd, opts=oracle_lib.default_opts(mode=md))[0]
            for md, sd in ((oracle_lib.MODE_CLE, 5), (oracle_lib.MODE_TAU_LEAP, 6))]
    for c in range(1, len(T)):
        a, b = runs[0][:, c, 0].astype(np.float64), runs[1][:, c, 0].astype(np.float64)
        se = np.sqrt(a.var() / n + b.var() / n)
        assert abs(a.mean() - b.mean()) < 4 * se
        assert abs(a.var() / b.var() - 1.0) < 4 * np.sqrt(4.0 / n)


def test_cle_equals_tau_leap_below_the_threshold(oracle_lib):
    b = inputs.random_batch(16, 32, 40, seed=71, t_end=10.0, n_samples=6, x0_max=100)
    a = oracle_lib.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=2,
                            opts=oracle_lib.default_opts(mode=oracle_lib.MODE_CLE, max_attempts=100_000))
    t = oracle_lib.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=2,
                            opts=oracle_lib.default_opts(max_attempts=100_000))
    assert np.array_equal(a[0], t[0])
    assert np.array_equal(a[1], t[1])
