"""Sweep histograms on the device (ssa_simulate_histograms_dev) equal the
histograms of the oracle's trajectories, count for count.

Per (sample time, species) cell the engine adds each recorded count to one of
n_bins uniform bins of width bin_width from bin_lo, with an underflow and an
overflow bin.  The reference here is the plain definition applied to the
oracle's trajectories (np.searchsorted on the bin edges), so any difference in
a trajectory or in the binning shows up as a differing count."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1309_7695_b300 import abi, inputs  # noqa: E402

DEV = torch.device("cuda:0")


def reference_histograms(samples, lo, width, n_bins):
    """counts[k, i, b] from trajectories [R, S, N]: bin 0 below lo, 1 + b for
    lo + b*width <= x < lo + (b+1)*width, n_bins + 1 from lo + n_bins*width on."""
    edges = lo + width * np.arange(n_bins + 1, dtype=np.int64)
    idx = np.searchsorted(edges, samples.astype(np.int64), side="right")   # 0 .. n_bins + 1
    R, S, N = samples.shape
    out = np.zeros((S, N, n_bins + 2), dtype=np.int64)
    for k in range(S):
        for i in range(N):
            out[k, i] = np.bincount(idx[:, k, i], minlength=n_bins + 2)
    return out


def gpu_histograms(batch, seed, lo, width, n_bins, counts=None, **opt):
    S, N = len(batch.sample_times), batch.network.n_species
    m = abi.Model(batch.network)
    if counts is None:
        counts = torch.zeros((S, N, n_bins + 2), dtype=torch.int64, device=DEV)
    st = torch.zeros((batch.n_sims, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)
    try:
        abi.ssa_simulate_histograms_dev(m, torch.from_numpy(batch.params).to(DEV), torch.from_numpy(batch.x0).to(DEV),
                                        batch.t_end, torch.from_numpy(batch.sample_times).to(DEV), counts, lo, width,
                                        n_bins, st, seed=seed, opts=abi.ssa_default_options(**opt))
        torch.cuda.synchronize()
    finally:
        m.close()
    return counts, st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)


@pytest.mark.parametrize("lo,width,n_bins", [(0, 50, 20), (100, 7, 13), (-5, 1000, 1)])
def test_histograms_equal_the_oracle_trajectories(lo, width, n_bins):
    b = inputs.random_batch(16, 32, 400, seed=43, t_end=20.0, n_samples=11)
    counts, st = gpu_histograms(b, 11, lo, width, n_bins, max_attempts=200_000)
    s, ost = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=11,
                             opts=oracle.default_opts(max_attempts=200_000))
    assert np.array_equal(counts.cpu().numpy(), reference_histograms(s, lo, width, n_bins))
    assert np.array_equal(st["firings"], ost["firings"])
    assert (counts.sum(dim=2) == b.n_sims).all()


def test_histograms_accumulate_over_batches_and_mm_conservation():
    # two launches into one array add up; E + ES = 200 in every Michaelis-Menten cell
    b = inputs.mm_batch(512, seed=5)
    counts, _ = gpu_histograms(b, 1, 0, 1, 201)
    counts, _ = gpu_histograms(b, 2, 0, 1, 201, counts=counts)
    s1, _ = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=1)
    s2, _ = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=2)
    want = reference_histograms(np.concatenate([s1, s2]), 0, 1, 201)
    got = counts.cpu().numpy()
    assert np.array_equal(got, want)
    # bin x + 1 of E holds the simulations with E = x, those have ES = 200 - x
    assert np.array_equal(got[:, 0, 1:202], got[:, 2, 1:202][:, ::-1])


def test_histogram_arguments_are_checked():
    b = inputs.mm_batch(4)
    m = abi.Model(b.network)
    args = (torch.from_numpy(b.params).to(DEV), torch.from_numpy(b.x0).to(DEV), b.t_end,
            torch.from_numpy(b.sample_times).to(DEV), torch.zeros((11, 4, 7), dtype=torch.int64, device=DEV))
    try:
        for lo, width, n_bins in [(0, 0, 5), (0, 1, 0)]:
            with pytest.raises(abi.SsaError) as e:
                abi.ssa_simulate_histograms_dev(m, *args, lo, width, n_bins)
            assert e.value.code == abi.SSA_EINVAL
    finally:
        m.close()
