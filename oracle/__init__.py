"""CPU oracle for the batched tau-leaping / SSA engine.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the benchmark's CPU-baseline leg, never by the engine.  It shares no code
with the CUDA path.

Contents
  tauleap_oracle.c  the algorithm in plain C (FP64, canonical operation order)
  cme.py            exact transient law of tiny closed systems (Chemical
                    Master Equation on a truncated state space)
  rre.py            reaction-rate equations (the deterministic mean-field
                    model) integrated with a library ODE solver
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MODE_TAU_LEAP = 0
MODE_EXACT_SSA = 1
MODE_CLE = 2   # tau-leaping with Langevin increments for leap means >= 1000
STATUS_NAMES = {0: "OK", 1: "STEP_LIMIT", 2: "OVERFLOW", 3: "REJECT_LIMIT", 4: "INVALID"}


class Opts(ctypes.Structure):
    """oracle_opts: the method's options (mode, n_c, eps, SSA fallback factor and block, retry and attempt caps)."""
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("n_c", ctypes.c_int32),
        ("eps", ctypes.c_double),
        ("ssa_factor", ctypes.c_double),
        ("ssa_block", ctypes.c_int32),
        ("max_halvings", ctypes.c_int32),
        ("max_attempts", ctypes.c_int64),
    ]


STATS_DTYPE = np.dtype([
    ("status", np.int32), ("reserved", np.int32), ("leaps", np.int64), ("rejected", np.int64),
    ("ssa_steps", np.int64), ("firings", np.int64), ("attempts", np.int64), ("t_final", np.float64),
])

_lib = None


def lib():
    """The oracle library.  ORACLE_LIBRARY, when set, names another build of
    the oracle's source to load instead (the mutation test uses it to run
    the pins against copies of the oracle with one planted mistake)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIBRARY") or _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_u01.restype = ctypes.c_double
        L.oracle_log.argtypes = [ctypes.c_double]
        L.oracle_log.restype = ctypes.c_double
        L.oracle_exp.argtypes = [ctypes.c_double]
        L.oracle_exp.restype = ctypes.c_double
        L.oracle_lnfact.argtypes = [ctypes.c_int64]
        L.oracle_lnfact.restype = ctypes.c_double
        L.oracle_poisson.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_poisson.restype = ctypes.c_int64
        for name in ("oracle_log_array", "oracle_exp_array"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            getattr(L, name).restype = None
        L.oracle_lnfact_array.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        L.oracle_lnfact_array.restype = None
        L.oracle_poisson_array.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_void_p]
        L.oracle_poisson_array.restype = None
        L.oracle_canon_sum.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.oracle_canon_sum.restype = ctypes.c_double
        L.oracle_canon_select.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double]
        L.oracle_canon_select.restype = ctypes.c_int32
        L.oracle_leap_quantities.argtypes = [ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 8 + [
            ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_leap_quantities.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = ctypes.c_int
        vp = ctypes.c_void_p
        L.oracle_simulate.argtypes = [
            ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp,
            ctypes.c_int64, vp, ctypes.c_int64, vp, vp, ctypes.c_double, vp, ctypes.c_int32,
            ctypes.c_uint64, ctypes.POINTER(Opts), vp, vp, ctypes.c_int]
        L.oracle_simulate.restype = ctypes.c_int
        L.oracle_rre.argtypes = [
            ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp,
            ctypes.c_int64, vp, vp, vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int64, vp, vp]
        L.oracle_rre.restype = ctypes.c_int
        L.oracle_normal_leap_array.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, vp]
        L.oracle_normal_leap_array.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of a 4-word counter under a 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(w0, w1):
    """The uniform (m + 1/2) 2^-52 of two Philox words, m their top 52 bits."""
    return lib().oracle_u01(w0, w1)


def log(x):
    """The canonical natural logarithm (Tang's table method)."""
    return lib().oracle_log(float(x))


def exp(x):
    """The canonical exponential (Cody-Waite reduction, Taylor polynomial)."""
    return lib().oracle_exp(float(x))


def lnfact(k):
    """The canonical ln k! (exact product below 10, Stirling's series above)."""
    return lib().oracle_lnfact(int(k))


def poisson(lam, seed, sim, attempt, j):
    """The canonical Poisson draw of reaction j at (simulation, attempt): inversion below 10, PTRS from 10."""
    return lib().oracle_poisson(float(lam), int(seed), int(sim), int(attempt), int(j))


def log_array(x):
    """log() of every element."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().oracle_log_array(_ptr(x), _ptr(y), x.size)
    return y


def exp_array(x):
    """exp() of every element."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().oracle_exp_array(_ptr(x), _ptr(y), x.size)
    return y


def lnfact_array(k):
    """lnfact() of every element."""
    k = np.ascontiguousarray(k, dtype=np.int64)
    y = np.empty(k.shape, dtype=np.float64)
    lib().oracle_lnfact_array(_ptr(k), _ptr(y), k.size)
    return y


def poisson_array(lam, n, seed=0):
    """n draws of Poisson(lam); draw i uses simulation index i (attempt 1, reaction 0)."""
    out = np.empty(int(n), dtype=np.int64)
    lib().oracle_poisson_array(float(lam), int(seed), int(n), _ptr(out))
    return out


def canon_sum(v):
    """The canonical sum of v: 32 lane-striped slots, then the xor-butterfly tree."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().oracle_canon_sum(_ptr(v), v.size)


def canon_select(v, u):
    """The canonical selection of an index with probability v[j] / canon_sum(v), given u in [0, 1)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    return int(lib().oracle_canon_select(_ptr(v), v.size, float(u)))


def leap_quantities(network, c, x, opts=None):
    """Propensities, critical flags, a0, a0c and tau' for one state."""
    csr = network.csr()
    N, M = network.n_species, network.n_reactions
    c = np.ascontiguousarray(c, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.int32)
    a = np.empty(M, dtype=np.float64)
    crit = np.empty(M, dtype=np.int32)
    sc = np.empty(3, dtype=np.float64)
    o = opts if opts is not None else default_opts()
    rc = lib().oracle_leap_quantities(
        N, M, _ptr(csr["react_ptr"]), _ptr(csr["react_species"]), _ptr(csr["react_coef"]),
        _ptr(csr["prod_ptr"]), _ptr(csr["prod_species"]), _ptr(csr["prod_coef"]),
        _ptr(c), _ptr(x), ctypes.byref(o), _ptr(a), _ptr(crit), _ptr(sc))
    if rc != 0:
        raise ValueError("invalid model")
    return {"a": a, "crit": crit.astype(bool), "a0": sc[0], "a0c": sc[1], "tau1": sc[2]}


def default_opts(mode=MODE_TAU_LEAP, eps=0.03, n_c=10, ssa_factor=10.0, ssa_block=100,
                 max_halvings=64, max_attempts=100_000_000) -> Opts:
    """Options with the method's default constants (CGP 2006's suggested SSA fallback values)."""
    return Opts(mode, n_c, eps, ssa_factor, ssa_block, max_halvings, max_attempts)


def simulate(network, params, x0, t_end, sample_times, seed=0, opts=None, sim_ids=None,
             sim_offset=0, threads=0):
    """Run simulations of ``network`` on the CPU.

    params [R, M] float64, x0 [R, N] int32, sample_times [S] float64.
    Row r uses the random stream of simulation ``sim_ids[r]`` (or
    ``sim_offset + r``).  Returns (samples [R, S, N] int32, stats [R]).
    """
    csr = network.csr()
    N, M = network.n_species, network.n_reactions
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, M)
    R = params.shape[0]
    x0 = np.ascontiguousarray(x0, dtype=np.int32).reshape(R, N)
    T = np.ascontiguousarray(sample_times, dtype=np.float64)
    S = int(T.shape[0])
    ids = None if sim_ids is None else np.ascontiguousarray(sim_ids, dtype=np.int64)
    samples = np.zeros((R, S, N), dtype=np.int32)
    stats = np.zeros(R, dtype=STATS_DTYPE)
    o = opts if opts is not None else default_opts()
    rc = lib().oracle_simulate(
        N, M, _ptr(csr["react_ptr"]), _ptr(csr["react_species"]), _ptr(csr["react_coef"]),
        _ptr(csr["prod_ptr"]), _ptr(csr["prod_species"]), _ptr(csr["prod_coef"]),
        R, _ptr(ids), int(sim_offset), _ptr(params), _ptr(x0), float(t_end), _ptr(T), S,
        int(seed), ctypes.byref(o), _ptr(samples), _ptr(stats), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the model (order > 2 or bad species index)")
    return samples, stats


def simulate_batch(batch, seed=0, opts=None, threads=0, rows=None):
    """Convenience wrapper over an ``inputs.Batch`` (optionally a subset of rows)."""
    if rows is None:
        return simulate(batch.network, batch.params, batch.x0, batch.t_end, batch.sample_times,
                        seed, opts, threads=threads)
    rows = np.asarray(rows, dtype=np.int64)
    return simulate(batch.network, batch.params[rows], batch.x0[rows], batch.t_end,
                    batch.sample_times, seed, opts, sim_ids=rows, threads=threads)


def num_threads() -> int:
    """OpenMP threads the oracle's batch entry points use."""
    return int(lib().oracle_num_threads())


__all__ = ["simulate", "simulate_batch", "philox", "log_array", "exp_array", "lnfact_array",
           "poisson_array", "canon_sum", "canon_select", "leap_quantities", "u01", "log", "exp", "lnfact", "poisson",
           "default_opts", "Opts", "STATS_DTYPE", "MODE_TAU_LEAP", "MODE_EXACT_SSA", "MODE_CLE",
           "STATUS_NAMES", "num_threads"]

_ = os  # keep import for path helpers used by build


def sample_moments(samples):
    """Per (sample time, species) mean and unbiased variance of the counts
    across simulations, from exact integer sums: with n simulations,
    S1 = sum x and S2 = sum x^2 (Python integers), mean = S1 / n and
    var = (n S2 - S1^2) / (n (n - 1)) (0 for n < 2), each converted to double
    once and divided once (correctly rounded, as the engine's sweep moments
    are defined).  samples: [n, S, N] int32."""
    x = np.asarray(samples)
    n = int(x.shape[0])
    S1 = x.astype(np.int64).sum(axis=0)
    S2 = (x.astype(object) ** 2).sum(axis=0)
    mean = np.empty(S1.shape, dtype=np.float64)
    var = np.zeros(S1.shape, dtype=np.float64)
    for idx in np.ndindex(S1.shape):
        s1 = int(S1[idx])
        mean[idx] = float(s1) / float(n)
        if n >= 2:
            var[idx] = float(n * int(S2[idx]) - s1 * s1) / float(n * (n - 1))
    return mean, var


def rre_simulate(network, params, x0, sample_times, rtol=1e-8, atol=1e-8, max_steps=1_000_000):
    """Deterministic reaction-rate-equation trajectories of a batch (the
    canonical Dormand-Prince 5(4) integration of oracle_rre): params [R, M],
    x0 [R, N] (counts, as initial concentrations), sample_times [S].
    Returns (states [R, S, N] float64, stats [R])."""
    csr = network.csr()
    N, M = network.n_species, network.n_reactions
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, M)
    x0 = np.ascontiguousarray(x0, dtype=np.int32).reshape(-1, N)
    T = np.ascontiguousarray(sample_times, dtype=np.float64)
    R, S = params.shape[0], len(T)
    out = np.zeros((R, S, N), dtype=np.float64)
    stats = np.zeros(R, dtype=STATS_DTYPE)
    rc = lib().oracle_rre(N, M, _ptr(csr["react_ptr"]), _ptr(csr["react_species"]), _ptr(csr["react_coef"]),
                          _ptr(csr["prod_ptr"]), _ptr(csr["prod_species"]), _ptr(csr["prod_coef"]),
                          R, _ptr(params), _ptr(x0), _ptr(T), S, float(rtol), float(atol), int(max_steps),
                          _ptr(out), _ptr(stats))
    if rc != 0:
        raise ValueError("invalid model")
    return out, stats


def normal_leap_array(lam, n, seed=0):
    """n Langevin increments of mean lam (streams sim = 0..n-1, attempt 1,
    reaction 0), as the CLE mode draws them for leap means >= 1000."""
    out = np.empty(n, dtype=np.int64)
    lib().oracle_normal_leap_array(float(lam), int(seed), int(n), _ptr(out))
    return out
