"""Sweep moments on the device (ssa_simulate_moments_dev) equal the moments
of the oracle's trajectories, bit for bit: both are fixed functions of exact
integer sums over the simulations."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1309_7695_b300 import abi, inputs  # noqa: E402


def _moments(batch, seed, opts):
    dev = torch.device("cuda:0")
    m = abi.Model(batch.network)
    S, N = len(batch.sample_times), batch.network.n_species
    mean = torch.full((S, N), -1.0, dtype=torch.float64, device=dev)
    var = torch.full((S, N), -1.0, dtype=torch.float64, device=dev)
    st = torch.zeros((batch.n_sims, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    try:
        abi.ssa_simulate_moments_dev(m, torch.from_numpy(batch.params).to(dev), torch.from_numpy(batch.x0).to(dev),
                                     batch.t_end, torch.from_numpy(batch.sample_times).to(dev), mean, var, st,
                                     seed=seed, opts=opts)
        torch.cuda.synchronize()
    finally:
        m.close()
    return mean.cpu().numpy(), var.cpu().numpy(), st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)


@pytest.mark.parametrize("n", [1, 2, 257])
def test_fp64_moments_equal_oracle_moments(n):
    b = inputs.random_batch(16, 32, n, seed=41, t_end=20.0, n_samples=11)
    o = abi.ssa_default_options(max_attempts=200_000)
    mean, var, st = _moments(b, 9, o)
    s, ost = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=9,
                             opts=oracle.default_opts(max_attempts=200_000))
    rm, rv = oracle.sample_moments(s)
    assert np.array_equal(mean, rm)
    assert np.array_equal(var, rv)
    assert np.array_equal(st["firings"], ost["firings"])


def test_fast_moments_equal_moments_of_fast_trajectories():
    b = inputs.random_batch(32, 64, 500, seed=42, t_end=10.0, n_samples=6)
    o = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=200_000)
    mean, var, _ = _moments(b, 3, o)
    dev = torch.device("cuda:0")
    m = abi.Model(b.network)
    out = torch.empty((b.n_sims, len(b.sample_times), b.network.n_species), dtype=torch.int32, device=dev)
    abi.ssa_simulate_dev(m, torch.from_numpy(b.params).to(dev), torch.from_numpy(b.x0).to(dev), b.t_end,
                         torch.from_numpy(b.sample_times).to(dev), out, None, seed=3, opts=o)
    torch.cuda.synchronize()
    m.close()
    rm, rv = oracle.sample_moments(out.cpu().numpy())
    assert np.array_equal(mean, rm)
    assert np.array_equal(var, rv)


def test_moments_reject_bad_arguments():
    b = inputs.random_batch(8, 16, 4, seed=43, t_end=5.0, n_samples=3)
    o = abi.ssa_default_options(layout=abi.SSA_LAYOUT_WARP)
    with pytest.raises(abi.SsaError):
        _moments(b, 1, o)
