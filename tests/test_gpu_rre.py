"""Batched reaction-rate-equation integration on the GPU
(ssa_integrate_rre_dev) against the oracle's canonical Dormand-Prince 5(4)
integration, bit for bit, on random networks, closed-form networks and the
step-limit path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1309_7695_b300 import abi, inputs  # noqa: E402


def gpu_rre(net, params, x0, T, **kw):
    dev = torch.device("cuda:0")
    params = np.ascontiguousarray(params, dtype=np.float64)
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    n = params.shape[0]
    m = abi.Model(net)
    out = torch.full((n, len(T), net.n_species), -7.0, dtype=torch.float64, device=dev)
    st = torch.zeros((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    try:
        abi.ssa_integrate_rre_dev(m, torch.from_numpy(params).to(dev), torch.from_numpy(x0).to(dev),
                                  torch.from_numpy(np.asarray(T, dtype=np.float64)).to(dev), out, st, **kw)
        torch.cuda.synchronize()
    finally:
        m.close()
    return out.cpu().numpy(), st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)


@pytest.mark.parametrize("N,M,n", [(8, 16, 40), (32, 64, 96), (40, 70, 33)])
def test_random_networks_bit_exact(N, M, n):
    b = inputs.random_batch(N, M, n, seed=61, t_end=10.0, n_samples=11, x0_max=500)
    got, gst = gpu_rre(b.network, b.params, b.x0, b.sample_times, rtol=1e-8, atol=1e-8, max_steps=200_000)
    ref, rst = oracle.rre_simulate(b.network, b.params, b.x0, b.sample_times, rtol=1e-8, atol=1e-8,
                                   max_steps=200_000)
    assert np.array_equal(got, ref)
    for f in ("status", "leaps", "rejected", "attempts", "t_final"):
        assert np.array_equal(gst[f], rst[f]), f


def test_isomerization_against_closed_form():
    net = inputs.isomerization()
    T = np.linspace(0.0, 10.0, 21)
    got, st = gpu_rre(net, [[0.7]] * 3, [[1000, 0]] * 3, T, rtol=1e-10, atol=1e-10)
    assert np.allclose(got[:, :, 0], 1000.0 * np.exp(-0.7 * T), rtol=1e-8, atol=1e-9)
    assert np.all(st["status"] == 0)


def test_step_limit_and_bad_arguments():
    b = inputs.random_batch(8, 16, 5, seed=62, t_end=50.0, n_samples=6, x0_max=100)
    got, st = gpu_rre(b.network, b.params, b.x0, b.sample_times, max_steps=3)
    ref, rst = oracle.rre_simulate(b.network, b.params, b.x0, b.sample_times, max_steps=3)
    assert np.array_equal(got, ref) and np.all(st["status"] == abi.SSA_STATUS_STEP_LIMIT)
    with pytest.raises(abi.SsaError):
        gpu_rre(b.network, b.params, b.x0, b.sample_times, rtol=0.0)
