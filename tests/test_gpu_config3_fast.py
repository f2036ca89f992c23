"""Fast mode on the 128 x 256 network at its full horizon, t_end = 100.

The configuration: the random network of 128 species and 256 reactions,
initial counts up to 10^4, judged on 8 fixed parameter sets.  Each set is
run with R = 1,000 coupled replicates (the same seeds, hence the same Philox
words) in fast mode and in the FP64 reference mode, attempt cap 2^22, and
compared per (sample time, species) cell with the criterion of
test_gpu_fast_mode.py: two-sample KS tests with a Holm correction at 0.01,
means within 1 % (means >= 10) and variances within 1 %, or within the
family-wise paired sampling error where 1 % is tighter than that.  R is
below the 10^4 of the configuration's text so that the pair of runs stays
within about two minutes (4,000 replicates took 500 s); the sampling-error
bounds scale with it.  Each set's report prints how many cells meet the bare
1 % variance bound.

Three of the sets are dominated by exact SSA blocks (about 10^6 SSA steps by
t = 30..70) and a replicate may reach the cap before t_end.  A capped
trajectory is a valid sample path up to its t_final, so a cell at sample
time T_k uses the replicate pairs whose t_final >= T_k in both modes (the
filter depends on the path only, so it keeps equal laws equal); the test
reports, per set, the fraction of pairs that reach t_end.

A direct leg compares fast mode with the oracle itself: 500 replicates of
the cheapest set (about 10^5 attempts each) run by the CPU oracle with the
same seeds, the same criterion."""
import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402
from test_gpu_fast_mode import moment_and_ks_report, run  # noqa: E402

N, M, T_END = 128, 256, 100.0
CAP = 1 << 22
SEED = 17


def sets():
    return inputs.random_batch(N, M, 8, seed=31, t_end=T_END, n_samples=11, x0_max=10_000)


def replicate(base, rows, reps):
    return inputs.Batch(base.network, np.repeat(base.params[rows], reps, axis=0),
                        np.repeat(base.x0[rows], reps, axis=0), T_END, base.sample_times)


def filtered_report(fast, fst, ref, rst, T, n_cells):
    """moment_and_ks_report over the sample times every used pair reaches:
    the cells at T_k use the pairs with t_final >= T_k in both modes."""
    reach = np.minimum(fst["t_final"], rst["t_final"])
    ok_status = np.isin(fst["status"], (0, 1)) & np.isin(rst["status"], (0, 1))   # OK or capped
    reports = []
    for k, tk in enumerate(T):
        use = ok_status & (reach >= tk)
        if use.sum() < 100:
            continue
        reports.append(moment_and_ks_report(fast[use][:, k:k + 1, :], ref[use][:, k:k + 1, :], n_cells))
    return reports, float((ok_status & (reach >= T_END)).mean())


def test_fast_matches_fp64_at_t100_on_eight_sets():
    base = sets()
    reps = 1000
    b = replicate(base, np.arange(8), reps)
    fast, fst = run(b, abi.SSA_FAST, seed=SEED, max_attempts=CAP)
    ref, rst = run(b, abi.SSA_FP64_REF, seed=SEED, max_attempts=CAP)
    assert fast.min() >= 0 and np.all(fast[:, 0, :] == b.x0)
    n_cells = 8 * len(b.sample_times) * N
    for s in range(8):
        sl = slice(s * reps, (s + 1) * reps)
        reps_, finished = filtered_report(fast[sl], fst[sl], ref[sl], rst[sl], b.sample_times, n_cells)
        assert len(reps_) >= 3, f"set {s}: fewer than 3 sample times reached by 100 pairs"
        ks = sum(r["ks_rejections"] for r in reps_)
        mean_ok = min(r["mean_ok"] for r in reps_)
        var_ok = min(r["var_ok"] for r in reps_)
        print(f"set {s}: {len(reps_)} sample times, finished {finished:.3f}, KS rejections {ks}, "
              f"max mean rel {max(r['max_mean_rel_ge_10'] for r in reps_):.4f}, "
              f"var within 1% {min(r['var_within_1pct'] for r in reps_):.3f}")
        assert ks == 0 and mean_ok == 1.0 and var_ok == 1.0, s


def test_fast_matches_the_oracle_directly_on_one_set():
    # set 5 is the cheapest at t_end = 100 (about 10^5 attempts per replicate)
    base = sets()
    reps = 500
    b = replicate(base, np.array([5]), reps)
    fast, fst = run(b, abi.SSA_FAST, seed=SEED, max_attempts=CAP)
    ref, rst = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=SEED,
                               opts=oracle.default_opts(max_attempts=CAP))
    ok = (fst["status"] == 0) & (rst["status"] == 0)
    assert ok.mean() > 0.99
    rep = moment_and_ks_report(fast[ok], ref[ok], len(b.sample_times) * N)
    print(f"set 5 vs oracle: {rep}")
    assert rep["ks_rejections"] == 0
    assert rep["mean_ok"] == 1.0 and rep["var_ok"] == 1.0
