"""Pins for the oracle's Poisson sampler (inversion below mean 10, PTRS at
and above): chi-square of draws against the exact Poisson pmf, plus moment
checks, on a grid of means that straddles the switch point."""
import numpy as np
import pytest
from scipy import stats

from conftest import chi2_pvalue


@pytest.mark.parametrize("lam,n", [
    (0.05, 200_000), (1.0, 200_000), (4.2, 200_000), (9.99, 300_000),
    (10.0, 300_000), (10.5, 300_000), (30.0, 300_000), (1000.0, 300_000),
])
def test_poisson_pmf_chi_square(oracle_lib, lam, n):
    k = oracle_lib.poisson_array(lam, n, seed=12345)
    assert k.min() >= 0
    lo, hi = int(k.min()), int(k.max())
    support = np.arange(lo, hi + 1)
    counts = np.bincount(k - lo, minlength=len(support))
    probs = stats.poisson.pmf(support, lam)
    # mass outside the observed range goes to the end bins
    probs[0] += stats.poisson.cdf(lo - 1, lam)
    probs[-1] += stats.poisson.sf(hi, lam)
    p = chi2_pvalue(counts, probs)
    assert p > 1e-3, (lam, p)


@pytest.mark.parametrize("lam", [0.1, 1.0, 9.99, 10.0, 30.0, 1000.0, 1e6])
def test_poisson_chi_square_and_ks_on_1e7_draws(oracle_lib, lam):
    # 10^7 draws per mean against the exact pmf (scipy): chi-square over the
    # support (bins of 100 values at 10^6), and the largest gap between the
    # empirical and the exact cdf, judged by the Kolmogorov law (conservative
    # for a discrete law)
    n = 10_000_000
    k = oracle_lib.poisson_array(lam, n, seed=2024)
    assert k.min() >= 0
    lo, hi = int(k.min()), int(k.max())
    support = np.arange(lo, hi + 1)
    counts = np.bincount(k - lo, minlength=len(support)).astype(np.float64)
    cdf = stats.poisson.cdf(support, lam)
    d = np.max(np.abs(np.cumsum(counts) / n - cdf))
    assert stats.kstwobign.sf(d * np.sqrt(n)) > 1e-3, (lam, d)
    if lam >= 1e5:
        edges = np.arange(lo, hi + 101, 100)
        counts = np.add.reduceat(counts, edges[:-1] - lo)
        probs = np.diff(stats.poisson.cdf(edges - 1, lam))
    else:
        probs = stats.poisson.pmf(support, lam)
    probs[0] += stats.poisson.cdf(lo - 1, lam)
    probs[-1] += stats.poisson.sf(support[-1] if lam < 1e5 else edges[-1] - 1, lam)
    assert chi2_pvalue(counts, probs) > 1e-3, lam


@pytest.mark.parametrize("lam", [0.3, 7.0, 12.0, 250.0, 1e6])
def test_poisson_moments(oracle_lib, lam):
    n = 200_000
    k = oracle_lib.poisson_array(lam, n, seed=777).astype(np.float64)
    se_mean = np.sqrt(lam / n)
    assert abs(k.mean() - lam) < 5 * se_mean
    # variance of the sample variance for Poisson: (mu4 - sigma^4)/n, mu4 = lam(1+3lam)
    se_var = np.sqrt((lam * (1 + 3 * lam) - lam * lam) / n)
    assert abs(k.var() - lam) < 5 * se_var


def test_poisson_large_mean_standardised(oracle_lib):
    lam = 1e6
    k = oracle_lib.poisson_array(lam, 100_000, seed=99).astype(np.float64)
    # compare against the exact Poisson cdf through binned probabilities
    edges = np.arange(lam - 5000, lam + 5001, 250.0)
    counts, _ = np.histogram(k, bins=edges)
    probs = np.diff(stats.poisson.cdf(edges - 1, lam))
    below = stats.poisson.cdf(edges[0] - 1, lam)
    above = stats.poisson.sf(edges[-1] - 1, lam)
    counts = np.concatenate([[np.sum(k < edges[0])], counts, [np.sum(k >= edges[-1])]])
    probs = np.concatenate([[below], probs, [above]])
    assert chi2_pvalue(counts, probs) > 1e-3


def test_poisson_zero_mean_and_streams(oracle_lib):
    assert oracle_lib.poisson(0.0, 1, 2, 3, 4) == 0
    # distinct (sim, attempt, j) give independent-looking draws; same inputs repeat
    a = [oracle_lib.poisson(5.0, 1, s, 1, 0) for s in range(50)]
    b = [oracle_lib.poisson(5.0, 1, s, 1, 0) for s in range(50)]
    c = [oracle_lib.poisson(5.0, 1, s, 1, 1) for s in range(50)]
    assert a == b
    assert a != c
