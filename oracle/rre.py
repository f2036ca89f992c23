"""Reaction-rate equations (TEST INFRASTRUCTURE).

The deterministic mean-field model of a mass-action network: the ODE system
dX/dt = sum_j nu_j a_j(X) with continuous X (Methods section: when species
are abundant the intrinsic fluctuations average out and X(t) follows the
reaction-rate equations; in the thermodynamic limit the stochastic and
mean-field models agree, Kurtz).  Integrated with scipy's adaptive RK45 at
tight tolerances; used to check that the stochastic mean approaches it as
molecule counts grow.

The stochastic 2X propensity c x(x-1)/2 has the mean-field form c x^2/2.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp


def integrate(network, rates, x0, times, rtol=1e-10, atol=1e-10):
    """Mean-field trajectory X(t) at `times` ([len(times), N]) by scipy's RK45."""
    nu = network.stoichiometry().astype(np.float64)  # [N, M]
    reactants = network.reactants
    rates = np.asarray(rates, dtype=np.float64)

    def rhs(_t, x):
        """dX/dt = nu a(X) with the mean-field rates."""
        a = np.empty(len(reactants))
        for j, row in enumerate(reactants):
            v = rates[j]
            for s, coef in row:
                v = v * (x[s] if coef == 1 else x[s] * x[s] / 2.0)
            a[j] = v
        return nu @ a

    times = np.asarray(times, dtype=np.float64)
    sol = solve_ivp(rhs, (0.0, float(times[-1])), np.asarray(x0, dtype=np.float64),
                    method="RK45", t_eval=times, rtol=rtol, atol=atol)
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.y.T  # [len(times), N]
