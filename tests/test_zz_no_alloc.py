"""The allocation-free entry point (ssa_simulate_dev_noalloc) gives the same
results as ssa_simulate_dev.

Some callers cannot allocate device memory: code running inside a memory
allocator's own callbacks, or programs that reserve all device memory up
front.  For them the library offers a launch path whose only scratch, the
kernel's work counter, sits in a static device array instead of a fresh
allocation.  This test calls it through the C ABI twice in a row (the array
keeps the previous call's contents, so the second call checks that it is
cleared) and compares with the allocating entry point, bit for bit as every
other parity test here does.  It lives in its own file, collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi, inputs  # noqa: E402


def _run(fn, model, batch, seed, layout):
    dev = torch.device("cuda:0")
    n, N, S = batch.n_sims, batch.network.n_species, len(batch.sample_times)
    p = torch.from_numpy(batch.params).to(dev)
    x = torch.from_numpy(batch.x0).to(dev)
    T = torch.from_numpy(batch.sample_times).to(dev)
    out = torch.full((n, S, N), -1, dtype=torch.int32, device=dev)
    st = torch.zeros((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    o = abi.ssa_default_options(max_attempts=100_000, layout=layout)
    fn(model, p, x, batch.t_end, T, out, st, seed=seed, opts=o)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("layout", [abi.SSA_LAYOUT_LANE, abi.SSA_LAYOUT_WARP], ids=["lane", "warp"])
def test_noalloc_matches_allocating_entry_point_twice(layout):
    batch = inputs.random_batch(16, 32, 300, seed=21, t_end=20.0, n_samples=11)
    model = abi.Model(batch.network)
    try:
        for seed in (5, 6):
            want = _run(abi.ssa_simulate_dev, model, batch, seed, layout)
            got1 = _run(abi.ssa_simulate_dev_noalloc, model, batch, seed, layout)
            got2 = _run(abi.ssa_simulate_dev_noalloc, model, batch, seed, layout)
            for got in (got1, got2):
                assert np.array_equal(got[0], want[0])
                assert np.array_equal(got[1], want[1])
            assert (want[0] >= 0).all()
    finally:
        model.close()
