"""The engine's device arithmetic, built for the host, against the oracle.

csrc/device_f64.cuh compiles for the host as well as the device (host code
takes portable equivalents of the bit intrinsics, with the same values).
This CPU test builds tests/devmath_host.cu with nvcc and checks the engine's
own ln, exp, ln k!, Philox, Poisson sampler (both its plain route and the
certified-FP32 route the lane kernels take) and Langevin increments against
the oracle's, bit for bit, over many inputs.  The GPU parity tests check the
same functions inside the kernels; this one reaches far more inputs."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dm(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("devmath") / "libdevmath_host.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
                    "-I", os.path.join(ROOT, "include"), "-o", out, os.path.join(ROOT, "tests", "devmath_host.cu")],
                   check=True)
    L = ctypes.CDLL(out)
    vp, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    for name in ("dm_log_array", "dm_exp_array", "dm_lnfact_array"):
        getattr(L, name).argtypes = [vp, vp, i64]
    L.dm_philox.argtypes = [vp, vp, vp]
    L.dm_poisson_array.argtypes = [f64, u64, i64, vp]
    L.dm_poisson_certified_array.argtypes = [f64, u64, i64, vp, vp]
    L.dm_normal_leap_array.argtypes = [f64, u64, i64, vp]
    for name in ("dm_f64_to_f32_array", "dm_f32_to_f64_array", "dm_floor_array", "dm_u53_array", "dm_small_array"):
        getattr(L, name).argtypes = [vp, vp, i64]
    L.dm_tau2_screen_array.argtypes = [vp, vp, vp, vp, i64]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_log_exp_lnfact_equal_the_oracle(dm, oracle_lib):
    rng = np.random.default_rng(81)
    x = np.concatenate([rng.random(200_000), np.exp(rng.uniform(-700, 700, 200_000)), 1 + rng.uniform(-1e-6, 1e-6, 50_000),
                        np.array([5e-324, 2.2e-308, 0.5, 1.0, 2.0, 1.7976931348623157e308])])
    y = np.empty_like(x)
    dm.dm_log_array(_p(x), _p(y), len(x))
    assert np.array_equal(y.view(np.int64), oracle_lib.log_array(x).view(np.int64))
    e = np.concatenate([rng.uniform(-745, 709, 200_000), -rng.uniform(0, 10, 100_000)])
    ye = np.empty_like(e)
    dm.dm_exp_array(_p(e), _p(ye), len(e))
    assert np.array_equal(ye.view(np.int64), oracle_lib.exp_array(e).view(np.int64))
    k = np.concatenate([np.arange(0, 5000), rng.integers(0, 2**40, 50_000)]).astype(np.int64)
    yk = np.empty(len(k))
    dm.dm_lnfact_array(_p(k), _p(yk), len(k))
    assert np.array_equal(yk.view(np.int64), oracle_lib.lnfact_array(k).view(np.int64))


def test_philox_equals_the_oracle(dm, oracle_lib):
    rng = np.random.default_rng(82)
    for _ in range(2000):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        dm.dm_philox(_p(ctr), _p(key), _p(out))
        assert out.tolist() == oracle_lib.philox(ctr.tolist(), key.tolist())


@pytest.mark.parametrize("lam", [1e-9, 0.003, 0.4, 1.0, 3.3, 9.999, 10.0, 10.5, 37.0, 999.0, 1.2e4, 3e6, 2.5e9])
def test_poisson_routes_equal_the_oracle(dm, oracle_lib, lam):
    n = 100_000
    ref = oracle_lib.poisson_array(lam, n, seed=5)
    a = np.empty(n, dtype=np.int64)
    dm.dm_poisson_array(lam, 5, n, _p(a))
    assert np.array_equal(a, ref)
    b = np.empty(n, dtype=np.int64)
    fb = ctypes.c_int64()
    dm.dm_poisson_certified_array(lam, 5, n, _p(b), ctypes.byref(fb))
    assert np.array_equal(b, ref)
    if lam < 10:
        assert fb.value < 0.002 * n    # the certified FP32 inversion decides nearly every draw


@pytest.mark.parametrize("lam", [1000.0, 4.4e4, 7e7])
def test_langevin_increments_equal_the_oracle(dm, oracle_lib, lam):
    n = 100_000
    a = np.empty(n, dtype=np.int64)
    dm.dm_normal_leap_array(lam, 9, n, _p(a))
    assert np.array_equal(a, oracle_lib.normal_leap_array(lam, n, seed=9))


@pytest.mark.parametrize("lam", [10.0, 11.7, 50.0, 123.4, 1000.0, 5003.3, 2.0e4, 65535.9, 65536.0, 1.0e5])
def test_ptrs_certified_iteration_equals_the_oracle(dm, oracle_lib, lam):
    # PTRS takes its candidate, squeeze and acceptance decisions in FP32 below
    # means of 2^16 and falls back to FP64 inside the margins: every draw must
    # still be the oracle's (three seeds, 300,000 draws each)
    for seed in (11, 12, 13):
        n = 100_000
        a = np.empty(n, dtype=np.int64)
        dm.dm_poisson_array(lam, seed, n, _p(a))
        assert np.array_equal(a, oracle_lib.poisson_array(lam, n, seed=seed))


def test_bit_assembled_conversions_equal_ieee(dm):
    # the kernels replace conversion instructions by integer bit assembly;
    # numpy's IEEE conversions are the reference (round to nearest even)
    rng = np.random.default_rng(83)
    bitsd = rng.integers(0, 2**63, 500_000, dtype=np.int64) | (rng.integers(0, 2, 500_000, dtype=np.int64) << 63)
    x = bitsd.view(np.float64)
    x = x[np.isfinite(x)]
    edge = np.array([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 1.1754943508222875e-38,
                     1.1754942106924411e-38, 2.0**-149, 1.5 * 2.0**-149, 1e-300, 1e300, 0.1, 1 + 2.0**-24,
                     1 + 3 * 2.0**-24, 1 + 2.0**-24 + 2.0**-50])
    x = np.concatenate([x, edge, np.exp(rng.uniform(-100, 100, 200_000)) * rng.choice([-1.0, 1.0], 200_000)])
    y = np.empty(len(x), dtype=np.float32)
    dm.dm_f64_to_f32_array(_p(x), _p(y), len(x))
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))
    f = rng.integers(0, 2**32, 500_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = f[np.isfinite(f)]
    yd = np.empty(len(f))
    dm.dm_f32_to_f64_array(_p(f), _p(yd), len(f))
    assert np.array_equal(yd.view(np.int64), f.astype(np.float64).view(np.int64))


def test_bit_assembled_floor_and_integer_conversions(dm):
    rng = np.random.default_rng(84)
    x = np.concatenate([rng.uniform(-1e6, 1e6, 300_000), rng.uniform(-3, 3, 100_000), np.round(rng.uniform(-1e9, 1e9, 10_000)),
                        np.array([-0.0, 0.0, -0.5, 0.5, -1.0, 2.0**52 + 1, -(2.0**52) - 1, 2.0**61, -(2.0**61)])])
    y = np.empty(len(x), dtype=np.int64)
    dm.dm_floor_array(_p(x), _p(y), len(x))
    assert np.array_equal(y, np.floor(x).astype(np.int64))
    v = np.concatenate([rng.integers(0, 2**53, 200_000, dtype=np.uint64), np.array([0, 1, 2**52, 2**53 - 1], dtype=np.uint64)])
    yu = np.empty(len(v))
    dm.dm_u53_array(_p(v), _p(yu), len(v))
    assert np.array_equal(yu, v.astype(np.float64))
    s = np.concatenate([rng.integers(-2**31 + 1, 2**31, 200_000), np.array([0, 1, -1, 2, -2, 127, -128])]).astype(np.int32)
    ys = np.empty(len(s))
    dm.dm_small_array(_p(s), _p(ys), len(s))
    assert np.array_equal(ys, s.astype(np.float64))


def test_tau2_screen_never_hides_a_critical_firing(dm, oracle_lib):
    # the leap drops tau'' = -ln(u)/a0c (Eq. 12's time to the next critical
    # firing) only when the FP32 screen says it exceeds m = min(tau', gap);
    # then the oracle's FP64 tau'' must exceed m too, or a critical firing the
    # oracle makes would be lost.  m is placed at and around the exact tau''.
    rng = np.random.default_rng(85)
    n = 400_000
    u = np.concatenate([rng.random(n // 4), 1 - rng.random(n // 4) * 2.0**-rng.integers(20, 53, n // 4),
                        np.exp(-rng.uniform(0, 740, n // 4)), rng.random(n // 4) * 2.0**-rng.integers(0, 127, n // 4)])
    # the screen's domain: u >= 2^-126, since every uniform is (m + 1/2) 2^-52
    assert oracle_lib.u01(0, 0) == 2.0**-53
    u = np.clip(u, 2.0**-126, np.nextafter(1.0, 0.0))
    a0c = np.exp(rng.uniform(-300, 300, n)) * rng.choice([1.0, 1e-10, 1e10], n)
    E = -oracle_lib.log_array(u)
    with np.errstate(over="ignore", under="ignore"):
        tau2 = E / a0c
    rel = np.concatenate([np.zeros(n // 4), rng.uniform(-1e-3, 1e-3, n // 4),
                          rng.uniform(-1e-6, 1e-6, n // 4), rng.uniform(-0.5, 0.5, n // 4)])
    with np.errstate(over="ignore", invalid="ignore"):
        m = tau2 * (1 + rel)
    m = np.where(rng.random(n) < 0.05, np.nextafter(tau2, 0.0), m)
    ok = np.isfinite(m) & (m > 0) & np.isfinite(tau2)
    u, a0c, m, tau2 = u[ok], a0c[ok], m[ok], tau2[ok]
    out = np.empty(len(u), dtype=np.uint8)
    dm.dm_tau2_screen_array(_p(u), _p(a0c), _p(m), _p(out), len(u))
    later = out.astype(bool)
    assert np.all(tau2[later] > m[later])
    # and it settles most cases that are not close: tau'' above 1.01 m with a0c
    # and tau'' in FP32 normal range and u not within 2^-18 of 1
    clear = (tau2 > 1.01 * m) & (a0c > 1e-37) & (a0c < 1e37) & (tau2 < 1e37) & (u < 1 - 2.0**-18) & (tau2 > 1e-30)
    assert clear.sum() > 5_000
    assert later[clear].mean() > 0.999


def test_philox_equals_the_oracle_on_1e9_words(oracle_lib, tmp_path):
    # the engine's Philox and the oracle's, written separately from the
    # published round function, agree word for word over 2.5e8 blocks
    from oracle import build as oracle_build

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = oracle_build.build()
    exe = str(tmp_path / "philox_words_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(ROOT, "tests", "philox_words_check.cu"),
                    "-L", os.path.dirname(lib), "-loracle", "-Xlinker", "-rpath=" + os.path.dirname(lib)], check=True)
    words, mismatches = (int(v) for v in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split())
    assert words == 10**9
    assert mismatches == 0


def test_certified_routes_equal_the_oracle_at_random_means(dm, oracle_lib):
    # the lane kernels' Poisson route (certified FP32 inversion, certified
    # PTRS iteration and acceptance, FP64 inside the margins) at 650 random
    # means from 1e-7 to 2^17, including the switch at 10 and the end of the
    # FP32 iteration at 2^16, 20,000 draws each, on random seeds
    rng = np.random.default_rng(86)
    lams = np.concatenate([np.exp(rng.uniform(np.log(1e-7), np.log(10.0), 200)),
                           np.exp(rng.uniform(np.log(10.0), np.log(2.0 ** 17), 400)),
                           rng.uniform(9.9, 10.0, 25), 2.0 ** 16 + rng.uniform(-50, 50, 25)])
    n = 20_000
    for lam in lams:
        seed = int(rng.integers(0, 2 ** 63))
        a = np.empty(n, dtype=np.int64)
        fb = ctypes.c_int64()
        dm.dm_poisson_certified_array(float(lam), seed, n, _p(a), ctypes.byref(fb))
        assert np.array_equal(a, oracle_lib.poisson_array(float(lam), n, seed=seed)), (lam, seed)
