"""The Langevin (CLE) mode on the GPU against the oracle, bit for bit:
networks whose leaps draw normal increments (leap means >= 1000) as well as
Poisson ones, the same Philox counters on both sides."""
import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402
from test_gpu_parity import assert_same, gpu_run  # noqa: E402


def _both(b, seed, cap):
    got = gpu_run(b, seed=seed, mode=abi.SSA_MODE_CLE, max_attempts=cap, layout=abi.SSA_LAYOUT_LANE)
    ref = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=seed,
                          opts=oracle.default_opts(mode=oracle.MODE_CLE, max_attempts=cap))
    return got, ref


def test_pure_production_normal_increments_bit_exact():
    net = inputs.Network(2, [[(0, 1)]], [[(0, 1), (1, 1)]])
    b = inputs.replicate_batch(net, [1.0], [1000, 0], 300, 4.0, 5)
    got, ref = _both(b, 3, 10_000)
    assert_same(got, ref, "pure production")
    assert np.all(got[1]["leaps"] == 4)


def test_birth_death_large_counts_bit_exact():
    b = inputs.replicate_batch(inputs.birth_death(), [2e5, 1.0], [0], 128, 5.0, 6)
    got, ref = _both(b, 5, 100_000)
    assert_same(got, ref, "birth-death")


def test_random_network_large_counts_bit_exact():
    b = inputs.random_batch(16, 32, 64, seed=72, t_end=2.0, n_samples=5, x0_max=100_000)
    got, ref = _both(b, 7, 50_000)
    assert_same(got, ref, "random network")


def test_cle_rejects_the_warp_layout():
    b = inputs.random_batch(8, 16, 4, seed=73, t_end=1.0, n_samples=3)
    with pytest.raises(abi.SsaError):
        gpu_run(b, mode=abi.SSA_MODE_CLE, layout=abi.SSA_LAYOUT_WARP)
