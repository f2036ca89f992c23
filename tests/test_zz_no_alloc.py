"""The allocation-free entry point (ssa_simulate_dev_noalloc) gives the same
results as ssa_simulate_dev, and allocates no device memory.

Some callers cannot allocate device memory: code running inside a memory
allocator's own callbacks, or programs that reserve all device memory up
front.  For them the library offers a launch path whose only scratch, the
kernel's work counter, sits in a static device array instead of a fresh
allocation.  This test calls it through the C ABI twice in a row (the array
keeps the previous call's contents, so the second call checks that it is
cleared) and compares with the allocating entry point, bit for bit as every
other parity test here does.  It also watches the device's default memory
pool, which serves the library's stream-ordered allocations: the no-alloc
calls must leave its high-water mark and its reserved size unchanged, while
the allocating entry point, as a control, does move the high-water mark.
(Torch's caching allocator does not draw on that pool.)  It lives in its own
file, collected last."""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi, inputs  # noqa: E402

POOL_RESERVED_CURRENT = 5   # cudaMemPoolAttrReservedMemCurrent
POOL_USED_CURRENT = 7       # cudaMemPoolAttrUsedMemCurrent
POOL_USED_HIGH = 8          # cudaMemPoolAttrUsedMemHigh


class DefaultPool:
    """The current device's default memory pool, through the CUDA runtime the
    library itself links (libcudart.so.13)."""

    def __init__(self):
        abi.lib()
        self.rt = ctypes.CDLL("libcudart.so.13", mode=ctypes.RTLD_GLOBAL)
        self.pool = ctypes.c_void_p()
        dev = ctypes.c_int()
        assert self.rt.cudaGetDevice(ctypes.byref(dev)) == 0
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, POOL_USED_HIGH, ctypes.byref(v)) == 0


def _run(fn, model, batch, seed, layout):
    dev = torch.device("cuda:0")
    n, N, S = batch.n_sims, batch.network.n_species, len(batch.sample_times)
    p = torch.from_numpy(batch.params).to(dev)
    x = torch.from_numpy(batch.x0).to(dev)
    T = torch.from_numpy(batch.sample_times).to(dev)
    out = torch.full((n, S, N), -1, dtype=torch.int32, device=dev)
    st = torch.zeros((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    o = abi.ssa_default_options(max_attempts=100_000, layout=layout)
    torch.cuda.synchronize()
    fn(model, p, x, batch.t_end, T, out, st, seed=seed, opts=o)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("layout", [abi.SSA_LAYOUT_LANE, abi.SSA_LAYOUT_WARP], ids=["lane", "warp"])
def test_noalloc_matches_allocating_entry_point_twice(layout):
    batch = inputs.random_batch(16, 32, 300, seed=21, t_end=20.0, n_samples=11)
    model = abi.Model(batch.network)
    pool = DefaultPool()
    try:
        for seed in (5, 6):
            # the no-alloc calls first, so that a first call on the device is covered too
            torch.cuda.synchronize()
            reserved = pool.get(POOL_RESERVED_CURRENT)
            used = pool.get(POOL_USED_CURRENT)
            pool.reset_high()   # the high-water mark restarts from the memory in use now
            got1 = _run(abi.ssa_simulate_dev_noalloc, model, batch, seed, layout)
            got2 = _run(abi.ssa_simulate_dev_noalloc, model, batch, seed, layout)
            assert pool.get(POOL_USED_HIGH) <= used, "the no-alloc path drew memory from the default pool"
            assert pool.get(POOL_RESERVED_CURRENT) <= reserved, "the no-alloc path grew the default pool"
            pool.reset_high()
            want = _run(abi.ssa_simulate_dev, model, batch, seed, layout)
            assert pool.get(POOL_USED_HIGH) > used, "control: the allocating entry point should use the pool"
            for got in (got1, got2):
                assert np.array_equal(got[0], want[0])
                assert np.array_equal(got[1], want[1])
            assert (want[0] >= 0).all()
    finally:
        model.close()


def test_noalloc_module_is_collected_last():
    here = os.path.dirname(os.path.abspath(__file__))
    later = [f for f in os.listdir(here) if f.startswith("test_") and f.endswith(".py") and f > "test_zz_no_alloc.py"]
    assert not later, later
