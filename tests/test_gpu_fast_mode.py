"""Fast mode (FP32 propensities, Poisson means and sampler; FP64 clock, a0
and tau selection) against the FP64 reference mode and exact laws.

Fast mode is not bit-exact by design; it is judged distributionally:
  - coupled runs (same seed, so the same Philox words) against the FP64
    reference, 8 parameter sets x 10^4 replicates: species means and
    variances at every sample time within 1 %, or within the family-wise
    sampling error of the paired difference where 1 % is below it, and
    two-sample KS tests at every sample time and species with a Holm
    correction at level 0.01;
  - the exact law where one is known (birth-death Poisson, the CME of a
    tiny closed system);
  - invariants (conservation, non-negative counts, the first sample)."""
import math

import numpy as np
import pytest
from scipy import stats

from conftest import chi2_pvalue
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402
from oracle import cme  # noqa: E402

DEV = torch.device("cuda:0")


def run(batch, precision, seed=0, mode=abi.SSA_MODE_TAU_LEAP, **opt):
    n, N, S = batch.n_sims, batch.network.n_species, len(batch.sample_times)
    m = abi.Model(batch.network)
    p = torch.from_numpy(np.ascontiguousarray(batch.params)).to(DEV)
    x = torch.from_numpy(np.ascontiguousarray(batch.x0)).to(DEV)
    T = torch.from_numpy(batch.sample_times).to(DEV)
    out = torch.empty((n, S, N), dtype=torch.int32, device=DEV)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)
    o = abi.ssa_default_options(precision=precision, mode=mode, **opt)
    abi.ssa_simulate_dev(m, p, x, batch.t_end, T, out, st, seed=seed, opts=o)
    torch.cuda.synchronize()
    m.close()
    return out.cpu().numpy(), st.cpu().numpy().view(abi.STATS_DTYPE).reshape(n)


def holm_reject(pvalues, alpha):
    p = np.sort(np.asarray(pvalues))
    m = len(p)
    for i, v in enumerate(p):
        if v > alpha / (m - i):
            return i          # number of rejections
    return m


def moment_and_ks_report(fast, ref, n_cells_total):
    """fast, ref: samples [R, S, N] of coupled replicates of one parameter set.

    Per (sample time, species) cell: mean within 1 % (means >= 10) and
    variance within 1 %; where the 1 % bound is tighter than the sampling
    error of the paired difference, within z* paired standard errors, z*
    the Bonferroni normal quantile at family-wise level 0.01 over all cells
    of the test.  Paired SEs come from per-replicate differences (identical
    coupled trajectories contribute zero): mean from f - r, variance from
    (f - mean_f)^2 - (r - mean_r)^2.  KS: two-sample tests at every cell with
    a Holm correction at 0.01.  Also reports how many cells meet the plain
    1 % variance bound and the fraction of identical trajectories."""
    R = fast.shape[0]
    f = fast.astype(np.float64)
    r = ref.astype(np.float64)
    mf, mr = f.mean(0), r.mean(0)
    vf, vr = f.var(0), r.var(0)
    se_m = (f - r).std(0) / math.sqrt(R)
    dv = (f - mf) ** 2 - (r - mr) ** 2
    se_v = dv.std(0) / math.sqrt(R)
    z = stats.norm.isf(0.01 / (2 * n_cells_total))
    big = np.abs(mr) >= 10
    mean_ok = np.abs(mf - mr) <= np.maximum(np.where(big, 0.01 * np.abs(mr), 0.0), z * se_m) + 1e-12
    var_strict = np.abs(vf - vr) <= 0.01 * vr + 1e-12
    var_ok = var_strict | (np.abs(vf - vr) <= z * se_v + 1e-12)
    pvals = []
    for s in range(f.shape[1]):
        for i in range(f.shape[2]):
            a, b = fast[:, s, i], ref[:, s, i]
            if a.min() == a.max() == b.min() == b.max():
                continue
            pvals.append(stats.ks_2samp(a, b).pvalue)
    same = float(np.mean((fast == ref).all(axis=(1, 2))))
    return {"mean_ok": float(mean_ok.mean()), "var_ok": float(var_ok.mean()),
            "var_within_1pct": float(var_strict.mean()), "var_within_1pct_mean_ge_10": float(var_strict[big].mean())
            if big.any() else 1.0, "max_mean_rel_ge_10": float((np.abs(mf - mr) / np.maximum(np.abs(mr), 1))[big].max())
            if big.any() else 0.0, "ks_rejections": holm_reject(pvals, 0.01),
            "ks_min_p": float(min(pvals)) if pvals else 1.0, "identical": same}


@pytest.mark.parametrize("N,M,t_end,x0max", [(32, 64, 20.0, 1000), (128, 256, 2.0, 10_000)])
def test_fast_matches_fp64_reference_coupled(N, M, t_end, x0max):
    # 8 fixed parameter sets x 10^4 replicates, same seed in both modes
    base = inputs.random_batch(N, M, 8, seed=31, t_end=t_end, n_samples=11, x0_max=x0max)
    reps = 10_000
    b = inputs.Batch(base.network, np.repeat(base.params, reps, axis=0), np.repeat(base.x0, reps, axis=0),
                     t_end, base.sample_times)
    fast, fst = run(b, abi.SSA_FAST, seed=17, max_attempts=1 << 18)
    ref, rst = run(b, abi.SSA_FP64_REF, seed=17, max_attempts=1 << 18)
    assert fast.min() >= 0
    assert np.all(fast[:, 0, :] == b.x0)
    n_cells = 8 * len(b.sample_times) * N
    reports = []
    for s in range(8):
        sl = slice(s * reps, (s + 1) * reps)
        ok = (fst["status"][sl] == 0) & (rst["status"][sl] == 0)
        rep = moment_and_ks_report(fast[sl][ok], ref[sl][ok], n_cells)
        rep["finished"] = float(ok.mean())
        print(f"{N}x{M} set {s}: {rep}")
        reports.append(rep)
    for rep in reports:
        assert rep["ks_rejections"] == 0, rep
        assert rep["mean_ok"] == 1.0 and rep["var_ok"] == 1.0, rep
    assert abs(fst["firings"].sum() / rst["firings"].sum() - 1) < 0.01


def test_fast_independent_seeds_within_sampling_error():
    base = inputs.random_batch(32, 64, 2, seed=32, t_end=10.0, n_samples=6)
    reps = 8000
    b = inputs.Batch(base.network, np.repeat(base.params, reps, 0), np.repeat(base.x0, reps, 0), 10.0,
                     base.sample_times)
    fast, _ = run(b, abi.SSA_FAST, seed=100, max_attempts=1 << 18)
    ref, _ = run(b, abi.SSA_FP64_REF, seed=200, max_attempts=1 << 18)
    for s in range(2):
        f = fast[s * reps:(s + 1) * reps].astype(float)
        r = ref[s * reps:(s + 1) * reps].astype(float)
        se = np.sqrt((f.var(0) + r.var(0)) / reps) + 1e-12
        z = np.abs(f.mean(0) - r.mean(0)) / se
        assert z.max() < 5.0


def test_fast_birth_death_law():
    times = [2.0, 5.0, 10.0, 30.0]
    b = inputs.replicate_batch(inputs.birth_death(), [10.0, 0.1], [0], 20_000, 30.0, 2)
    b.sample_times = np.asarray(times)
    s, st = run(b, abi.SSA_FAST, seed=1)
    assert np.all(st["status"] == 0)
    for q, t in enumerate(times):
        lam = 100.0 * (1.0 - math.exp(-0.1 * t))
        x = s[:, q, 0]
        sup = np.arange(x.max() + 1)
        pr = stats.poisson.pmf(sup, lam)
        pr[-1] += stats.poisson.sf(x.max(), lam)
        assert chi2_pvalue(np.bincount(x, minlength=len(sup)), pr) > 1e-3


@pytest.mark.parametrize("mode", [abi.SSA_MODE_EXACT, abi.SSA_MODE_TAU_LEAP], ids=["exact", "tau"])
def test_fast_tiny_michaelis_menten_matches_cme(mode):
    net, rates, x0, times = inputs.michaelis_menten(), [1.0, 0.5, 0.7], [2, 3, 0, 0], [0.3, 1.0, 3.0]
    states, probs = cme.transient_distribution(net, rates, x0, times)
    b = inputs.replicate_batch(net, rates, x0, 40_000, 3.0, 2)
    b.sample_times = np.asarray(times)
    s, _ = run(b, abi.SSA_FAST, seed=4, mode=mode)
    lookup = {tuple(v): i for i, v in enumerate(states)}
    for q in range(len(times)):
        idx = np.array([lookup[tuple(v)] for v in s[:, q, :]])
        assert chi2_pvalue(np.bincount(idx, minlength=len(states)), probs[q]) > 1e-3


def test_fast_invariants_mm_sweep():
    b = inputs.mm_batch(1024, seed=2)
    s, st = run(b, abi.SSA_FAST, seed=3)
    assert np.all(st["status"] == 0)
    assert np.all(s[:, :, 0] + s[:, :, 2] == 200)
    assert np.all(s[:, :, 1] + s[:, :, 2] + s[:, :, 3] == 500)
    assert np.all(s[:, 0, :] == b.x0)


def test_fast_rejects_warp_layout():
    b = inputs.mm_batch(4)
    with pytest.raises(abi.SsaError) as e:
        run(b, abi.SSA_FAST, layout=abi.SSA_LAYOUT_WARP)
    assert e.value.code == abi.SSA_EUNSUPPORTED
