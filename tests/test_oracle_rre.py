"""The oracle's deterministic reaction-rate-equation integrator against
closed-form solutions and against scipy's RK45 (an independent adaptive
integrator) on random networks."""
import math

import numpy as np

from paper_1309_7695_b300 import inputs


def test_isomerization_exponential_decay(oracle_lib):
    net = inputs.isomerization()          # A -> B, rate k
    k, A0 = 0.7, 1000
    T = np.linspace(0.0, 10.0, 41)
    out, st = oracle_lib.rre_simulate(net, [[k]], [[A0, 0]], T, rtol=1e-10, atol=1e-10)
    exact = A0 * np.exp(-k * T)
    assert np.allclose(out[0, :, 0], exact, rtol=1e-8, atol=1e-9)
    assert np.allclose(out[0, :, 0] + out[0, :, 1], A0, rtol=1e-12)     # conservation
    assert st["status"][0] == 0 and st["leaps"][0] > 0


def test_birth_death_relaxation(oracle_lib):
    net = inputs.birth_death()            # 0 -> X (k), X -> 0 (g)
    k, g, x0 = 10.0, 0.1, 5
    T = np.linspace(0.0, 60.0, 31)
    out, _ = oracle_lib.rre_simulate(net, [[k, g]], [[x0]], T, rtol=1e-10, atol=1e-10)
    exact = k / g + (x0 - k / g) * np.exp(-g * T)
    assert np.allclose(out[0, :, 0], exact, rtol=1e-8)


def test_dimerization_closed_form(oracle_lib):
    net = inputs.dimerization()           # 2A -> B: dA/dt = -2 (c A^2 / 2) = -c A^2
    c = 0.01
    row = [r for r in net.reactants]
    M = net.n_reactions
    params = np.zeros((1, M))
    params[0, 0] = c                       # only the forward dimerization
    x0 = np.zeros((1, net.n_species), dtype=np.int32)
    x0[0, 0] = 400
    T = np.linspace(0.0, 5.0, 21)
    out, _ = oracle_lib.rre_simulate(net, params, x0, T, rtol=1e-10, atol=1e-10)
    assert row[0] == [(0, 2)] or sorted(row[0]) == [(0, 2)]
    exact = 400.0 / (1.0 + c * 400.0 * T)
    assert np.allclose(out[0, :, 0], exact, rtol=1e-8)


def test_random_networks_match_scipy_rk45(oracle_lib):
    from oracle import rre

    b = inputs.random_batch(8, 16, 6, seed=51, t_end=5.0, n_samples=11, x0_max=200)
    out, st = oracle_lib.rre_simulate(b.network, b.params, b.x0, b.sample_times, rtol=1e-10, atol=1e-10)
    for r in range(b.n_sims):
        ref = rre.integrate(b.network, b.params[r], b.x0[r], b.sample_times, rtol=1e-11, atol=1e-11)
        scale = np.maximum(np.abs(ref), 1.0)
        assert np.all(np.abs(out[r] - ref) <= 1e-6 * scale), r
        assert st["status"][r] == 0


def test_step_limit_and_first_sample(oracle_lib):
    b = inputs.random_batch(8, 16, 3, seed=52, t_end=50.0, n_samples=6, x0_max=100)
    out, st = oracle_lib.rre_simulate(b.network, b.params, b.x0, b.sample_times, max_steps=3)
    assert np.all(st["status"] == 1)
    assert np.all(st["leaps"] + st["rejected"] == 3)
    assert np.array_equal(out[:, 0, :], b.x0.astype(np.float64))   # T[0] = 0 records x0
    # after the stop, every later sample repeats the last state
    assert np.array_equal(out[:, -1, :], out[:, -2, :])
    assert math.isfinite(float(out.sum()))
