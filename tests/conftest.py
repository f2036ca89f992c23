"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device (the parity tests of the engine against the
          oracle).  Everything else runs on the CPU.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (engine parity and GPU checks)")


def chi2_pvalue(observed_counts, expected_probs, min_expected=5.0):
    """Pearson chi-square p-value, merging sparse bins into their neighbours."""
    from scipy import stats

    obs = np.asarray(observed_counts, dtype=np.float64)
    p = np.asarray(expected_probs, dtype=np.float64)
    n = obs.sum()
    exp = p / p.sum() * n
    order = np.argsort(-exp)
    obs, exp = obs[order], exp[order]
    merged_o, merged_e = [], []
    acc_o = acc_e = 0.0
    for o, e in zip(obs, exp):
        acc_o += o
        acc_e += e
        if acc_e >= min_expected:
            merged_o.append(acc_o)
            merged_e.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 and merged_e:
        merged_o[-1] += acc_o
        merged_e[-1] += acc_e
    merged_o = np.asarray(merged_o)
    merged_e = np.asarray(merged_e)
    stat = ((merged_o - merged_e) ** 2 / merged_e).sum()
    dof = max(len(merged_e) - 1, 1)
    return float(stats.chi2.sf(stat, dof))


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.lib()
    return oracle
