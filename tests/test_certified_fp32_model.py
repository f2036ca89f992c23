"""The FP32 margins behind the engine's certified decisions, checked on a
float32 model.

The FP64 reference kernels decide the Poisson inversion (u <= F(k)) and the
PTRS acceptance test after the squeeze first in FP32, and fall back to the
exact FP64 evaluation only when the FP32 value lies within a stated margin
of the decision boundary; the margins are derived from the rounding of each
operation and the documented accuracy of expf / logf.  Here the same FP32
arithmetic is replayed with numpy float32 (its exp / log are of comparable
accuracy) against the canonical FP64 values, and every decision the model
calls certain must be the canonical one.  The fallback rate is reported as
the share of ambiguous cases, which must stay small for the fast path to
pay.  The kernels' own decisions are checked bit for bit by the GPU parity
tests."""
import math

import numpy as np

f32 = np.float32


def canonical_inversion(lam, u, exp):
    # the canonical search: p0 = exp(-lam), p_k = (p_{k-1} lam) (1/k), stop when u <= F
    # or when a term no longer changes F, at most 100 terms
    p = exp(-lam)
    F = p
    k = 0
    while u > F and k < 100:
        k += 1
        p = (p * lam) * (1.0 / k)
        Fn = F + p
        if Fn == F:
            break
        F = Fn
    return k


def certified_inversion_model(lam, u):
    lf, uf = f32(lam), f32(u)
    p = f32(np.exp(-lf))
    F = p
    for k in range(40):
        m = f32(4e-6) + f32(6e-7) * f32(k)
        if uf <= F - m:
            return k
        if not (uf > F + m):
            return -1
        p = f32(f32(p * lf) / f32(k + 1))
        F = f32(F + p)
    return -1


def canonical_cdf(lam, k, exp):
    p = exp(-lam)
    F = p
    for i in range(1, k + 1):
        p = (p * lam) * (1.0 / i)
        F = F + p
    return F


def test_certified_inversion_agrees_with_canonical(oracle_lib):
    rng = np.random.default_rng(21)
    lams = np.concatenate([rng.uniform(0.0, 10.0, 30_000), np.exp(rng.uniform(-20, 2.3, 10_000))])
    lams = lams[(lams > 0) & (lams < 10)]
    us = rng.random(len(lams))
    amb_random = 0
    for i, (lam, u) in enumerate(zip(lams, us)):
        lam, u = float(lam), float(u)
        cases = [u]
        if i % 5 == 0:   # uniforms exactly at a cdf value and one ulp above it
            F = canonical_cdf(lam, int(rng.integers(0, 8)), oracle_lib.exp)
            if 0 < F < 1:
                cases += [F, float(np.nextafter(F, 2.0))]
        for c, uu in enumerate(cases):
            k_ref = canonical_inversion(lam, uu, oracle_lib.exp)
            k = certified_inversion_model(lam, uu)
            if k < 0:
                amb_random += (c == 0)
            else:
                assert k == k_ref, (lam, uu, k, k_ref)
    # boundary uniforms must fall back (or be right); random ones almost never fall back
    assert amb_random / len(lams) < 2e-3


def certified_ptrs_model(lam, k, V, us, a, b):
    if not lam < 2.0 ** 22:
        return 0
    lf, kf, af, bf, usf, Vf = (f32(v) for v in (lam, k, a, b, us, V))
    inv_alpha = f32(f32(1.1239) + f32(f32(1.1328) / f32(bf - f32(3.4))))
    lhs = f32(np.log(f32(f32(Vf * inv_alpha) / f32(f32(af / f32(usf * usf)) + bf))))
    # log_pmf_f32
    if kf < 10:
        fact = f32(math.factorial(int(kf)))
        rhs = f32(f32(kf * np.log(lf)) - lf) - np.log(fact)
    else:
        d = f32(kf - lf)
        v = f32(d / f32(kf + lf))
        if abs(v) < 0.25:
            v2 = f32(v * v)
            s = f32(1.0 / 15.0)
            for c in (13, 11, 9, 7, 5, 3):
                s = f32(f32(s * v2) + f32(1.0 / c))
            D = f32(f32(v * d) + f32(f32(f32(2.0) * kf) * f32(f32(v * v2) * s)))
        else:
            D = f32(f32(kf * np.log(f32(kf / lf))) + lf) - kf
        rk = f32(f32(1.0) / kf)
        corr = f32(rk * f32(f32(1.0 / 12.0) - f32(f32(rk * rk) * f32(1.0 / 360.0))))
        rhs = f32(f32(-D - f32(f32(0.5) * np.log(f32(f32(6.283185307) * kf)))) - corr)
    d = abs(f32(kf - lf))
    m = f32(5e-5) + f32(4e-6) * f32(abs(rhs) + d)
    if k < 10:
        m += f32(2.0 ** -20) * lf
    elif d >= 0.25 * (kf + lf):
        m += f32(4e-6) * kf * abs(np.log(f32(kf / lf)))
    if lhs < rhs - m:
        return 1
    if lhs > rhs + m:
        return -1
    return 0


def test_certified_ptrs_acceptance_agrees_with_fp64():
    rng = np.random.default_rng(22)
    n_slow = n_amb = 0
    for lam in np.exp(rng.uniform(math.log(10.0), math.log(2.0 ** 22), 4000)):
        slam = math.sqrt(lam)
        b = 0.931 + 2.53 * slam
        a = -0.059 + 0.02483 * b
        vr = 0.9277 - 3.6224 / (b - 2.0)
        inv_alpha = 1.1239 + 1.1328 / (b - 3.4)
        for _ in range(60):
            U = rng.random() - 0.5
            V = rng.random()
            us = 0.5 - abs(U)
            if us <= 0 or V <= 0:
                continue
            k = math.floor((2.0 * a / us + b) * U + lam + 0.43)
            if us >= 0.07 and V <= vr:
                continue
            if k < 0 or (us < 0.013 and V > us):
                continue
            lhs = math.log(V * inv_alpha / (a / (us * us) + b))
            rhs = -lam + k * math.log(lam) - math.lgamma(k + 1.0)
            dec = certified_ptrs_model(lam, k, V, us, a, b)
            n_slow += 1
            if dec == 0:
                n_amb += 1
            else:
                assert (dec > 0) == (lhs <= rhs), (lam, k, lhs, rhs)
    assert n_slow > 10_000
    assert n_amb / n_slow < 1e-2


def ssa_screen_model(net, a, crit, x, a0, eps=0.03, ssa_factor=10.0):
    """float32 replay of the kernels' screen: True when an FP32 upper bound of
    tau' lies below an FP32 lower bound of ssa_factor / a0."""
    nu = net.stoichiometry()
    N, M = nu.shape
    irs = np.zeros(N, dtype=bool)
    hor = np.zeros(N, dtype=int)
    for j, row in enumerate(net.reactants):
        coefs = {}
        for s, c in row:
            coefs[s] = coefs.get(s, 0) + c
        order = sum(coefs.values())
        for s, c in coefs.items():
            hor[s] = max(hor[s], 3 if c == 2 else order)
            if not crit[j]:
                irs[s] = True
    qmin = np.float32(np.inf)
    for i in range(N):
        if not irs[i]:
            continue
        muf = s2f = absf = f32(0.0)
        n = 0
        for j in range(M):
            if nu[i, j] == 0 or crit[j] or not a[j] > 0:
                continue
            af, nvf = f32(a[j]), f32(nu[i, j])
            muf = f32(muf + f32(nvf * af))
            s2f = f32(s2f + f32(f32(nvf * nvf) * af))
            absf = f32(absf + f32(abs(nvf) * af))
            n += 1
        if n == 0:
            continue
        xf = f32(x[i])
        bf = f32(f32(eps) * xf)
        if hor[i] == 2 or (hor[i] != 1 and x[i] < 2):
            bf = f32(bf * f32(0.5))
        elif hor[i] != 1:
            bf = f32(bf / f32(f32(2.0) + f32(f32(1.0) / f32(xf - f32(1.0)))))
        bf = f32(max(bf, f32(1.0)) * f32(1.000001))
        err = f32(f32(n + 4) * f32(2.0 ** -20) * absf)
        amu = abs(muf)
        if amu > f32(2.0) * err:
            qmin = min(qmin, f32(f32(bf * f32(1.0001)) / f32(amu - err)))
        q2 = f32(f32(f32(bf * bf) * f32(1.0002)) / f32(s2f * f32(f32(1.0) - f32(n + 4) * f32(2.0 ** -20))))
        if q2 > 0:
            qmin = min(qmin, q2)
    thr_lo = f32(f32(f32(ssa_factor) / f32(a0)) * f32(0.9999))
    return bool(qmin < thr_lo)


def test_ssa_screen_never_contradicts_the_canonical_decision(oracle_lib):
    from paper_1309_7695_b300 import inputs

    rng = np.random.default_rng(23)
    certain = total = 0
    for net_seed, (N, M) in enumerate([(8, 16), (32, 64), (64, 128)]):
        net = inputs.random_network(N, M, 300 + net_seed)
        for _ in range(300):
            c = inputs.log_uniform(rng, 1e-4, 1.0, M)
            x = rng.integers(0, [12, 200, 5000][rng.integers(3)], size=N).astype(np.int32)
            q = oracle_lib.leap_quantities(net, c, x)
            if not q["a0"] > 0:
                continue
            total += 1
            if ssa_screen_model(net, q["a"], q["crit"], x, q["a0"]):
                certain += 1
                assert q["tau1"] < 10.0 / q["a0"], (net_seed, q["tau1"], 10.0 / q["a0"])
    assert total > 500
    assert certain > 0.2 * total   # the screen settles a good share of SSA decisions


def tau2_screen_model(u, a0c, m):
    """float32 replay of the screen that skips tau'' = -ln(u)/a0c when it is
    certainly larger than m = min(tau', delta)."""
    a0cf = f32(a0c)
    Ef = -np.log(f32(u))
    lo = f32(max(f32(Ef * f32(0.9999)) - f32(2.0 ** -20), f32(0.0)) / f32(a0cf * f32(1.0001)))
    return bool(a0cf >= f32(2.0 ** -126) and lo <= f32(2.0 ** 127) and float(lo) > m)


def test_tau2_screen_is_a_lower_bound(oracle_lib):
    rng = np.random.default_rng(24)
    n = 200_000
    u = rng.random(n)
    u[:1000] = 1.0 - rng.random(1000) * 2.0 ** -30        # -ln u tiny
    a0c = np.exp(rng.uniform(-30, 30, n))
    tau2 = -oracle_lib.log_array(u) / a0c                 # canonical E / a0c
    m = tau2 * np.exp(rng.normal(0.0, 1e-3, n))           # thresholds close to tau''
    skipped = 0
    for i in range(n):
        if tau2_screen_model(u[i], a0c[i], m[i]):
            skipped += 1
            assert tau2[i] > m[i], (u[i], a0c[i], m[i])
    assert skipped > 0.3 * n
