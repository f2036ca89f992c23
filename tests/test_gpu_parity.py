"""Parity of the CUDA engine (FP64 reference mode) with the CPU oracle.

The bar is bit-exactness: identical int32 trajectories at every sample time,
identical per-simulation counters and status, and identical t_final bits.
Both sides consume the same Philox counters and perform the same IEEE
operations in the same order, so any difference is a bug on one side."""
import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402

DEV = torch.device("cuda:0")
LAYOUTS = [abi.SSA_LAYOUT_LANE, abi.SSA_LAYOUT_WARP]
LAYOUT_IDS = ["lane", "warp"]


def gpu_run(batch, seed=0, mode=abi.SSA_MODE_TAU_LEAP, sim_offset=0, rows=None, **opt):
    params = batch.params if rows is None else batch.params[rows]
    x0 = batch.x0 if rows is None else batch.x0[rows]
    n, N, S = params.shape[0], batch.network.n_species, len(batch.sample_times)
    m = abi.Model(batch.network)
    p = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    x = torch.from_numpy(np.ascontiguousarray(x0)).to(DEV)
    T = torch.from_numpy(np.ascontiguousarray(batch.sample_times)).to(DEV)
    out = torch.full((n, S, N), -7, dtype=torch.int32, device=DEV)
    st = torch.zeros((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)
    o = abi.ssa_default_options(mode=mode, **opt)
    abi.ssa_simulate_dev(m, p, x, batch.t_end, T, out, st, seed=seed, opts=o, sim_offset=sim_offset)
    torch.cuda.synchronize()
    stats = st.cpu().numpy().view(abi.STATS_DTYPE).reshape(n)
    m.close()
    return out.cpu().numpy(), stats


def oracle_run(batch, seed=0, mode=oracle.MODE_TAU_LEAP, rows=None, sim_offset=0, **opt):
    o = oracle.default_opts(mode=mode, **opt)
    if rows is None:
        return oracle.simulate(batch.network, batch.params, batch.x0, batch.t_end, batch.sample_times,
                               seed=seed, opts=o, sim_offset=sim_offset)
    ids = np.asarray(rows, dtype=np.int64) + sim_offset
    return oracle.simulate(batch.network, batch.params[rows], batch.x0[rows], batch.t_end,
                           batch.sample_times, seed=seed, opts=o, sim_ids=ids)


def assert_same(gpu, ref, what=""):
    gs, gst = gpu
    rs, rst = ref
    assert gs.shape == rs.shape
    bad = np.argwhere((gs != rs).any(axis=(1, 2)))
    assert bad.size == 0, f"{what}: trajectories differ for sims {bad[:8].ravel().tolist()}"
    for f in ("status", "leaps", "rejected", "ssa_steps", "firings", "attempts"):
        assert np.array_equal(gst[f], rst[f]), (what, f, np.argwhere(gst[f] != rst[f])[:5].ravel())
    assert np.array_equal(gst["t_final"].view(np.int64), rst["t_final"].view(np.int64)), what


# ------------------------------------------------------------- workloads

@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
@pytest.mark.parametrize("mode", [abi.SSA_MODE_EXACT, abi.SSA_MODE_TAU_LEAP], ids=["exact", "tau"])
def test_michaelis_menten_sweep_bit_exact(mode, layout):
    b = inputs.mm_batch(1024, seed=0)
    assert_same(gpu_run(b, seed=0, mode=mode, layout=layout), oracle_run(b, seed=0, mode=mode), "MM")


@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
def test_michaelis_menten_large_counts_leaps_bit_exact(layout):
    b = inputs.mm_batch(256, seed=1, scale=100.0)
    ref = oracle_run(b, seed=3, eps=0.03)
    assert ref[1]["leaps"].sum() > 0
    assert_same(gpu_run(b, seed=3, eps=0.03, layout=layout), ref, "MM x100")


@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
@pytest.mark.parametrize("N,M,n,t_end,cap", [
    (32, 64, 320, 100.0, 200_000),     # the 32 x 64 sweep shape, 10 tiles of 32 sims
    (128, 256, 40, 20.0, 100_000),     # the 128 x 256 shape (N, M > 32: several lanes' chunks)
    (5, 7, 333, 50.0, 200_000),        # ragged: M, N not multiples of 32
    (40, 33, 97, 30.0, 200_000),       # M = 33: one full chunk + 1
])
def test_random_network_bit_exact(N, M, n, t_end, cap, layout):
    b = inputs.random_batch(N, M, n, seed=11, t_end=t_end, n_samples=21,
                            x0_max=1000 if N <= 32 else 10_000)
    ref = oracle_run(b, seed=5, max_attempts=cap)
    got = gpu_run(b, seed=5, max_attempts=cap, layout=layout)
    assert_same(got, ref, f"random {N}x{M}")
    assert ref[1]["leaps"].sum() > 0 and ref[1]["ssa_steps"].sum() > 0


@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
def test_closed_form_networks_bit_exact(layout):
    cases = [
        (inputs.birth_death(), [10.0, 0.1], [0], 30.0),
        (inputs.isomerization(), [1.0], [10_000, 0], 2.0),
        (inputs.dimerization(), [0.01, 0.5], [3000, 0], 5.0),
        (inputs.Network(2, [[(0, 1)]], [[(0, 1), (1, 1)]]), [0.7], [20, 0], 4.0),
    ]
    for net, rates, x0, t_end in cases:
        b = inputs.replicate_batch(net, rates, x0, 200, t_end, 7)
        for mode in (abi.SSA_MODE_EXACT, abi.SSA_MODE_TAU_LEAP):
            assert_same(gpu_run(b, seed=2, mode=mode, layout=layout), oracle_run(b, seed=2, mode=mode),
                        net.name)


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
def test_status_paths_bit_exact(layout):
    # step cap, overflow (A -> 2A explodes), frozen system, in both modes
    for mode in (abi.SSA_MODE_TAU_LEAP, abi.SSA_MODE_EXACT):
        b = inputs.random_batch(8, 16, 64, seed=4, t_end=50.0, n_samples=11)
        assert_same(gpu_run(b, max_attempts=37, layout=layout, mode=mode),
                    oracle_run(b, max_attempts=37, mode=mode), "cap")
        boom = inputs.replicate_batch(inputs.Network(1, [[(0, 1)]], [[(0, 2)]]), [1.0], [1000], 16, 100.0, 11)
        cap = 1 << 22 if mode == abi.SSA_MODE_TAU_LEAP else 1 << 14   # exact SSA: one birth per step
        got = gpu_run(boom, layout=layout, mode=mode, max_attempts=cap)
        want = abi.SSA_STATUS_OVERFLOW if mode == abi.SSA_MODE_TAU_LEAP else abi.SSA_STATUS_STEP_LIMIT
        assert np.all(got[1]["status"] == want)
        assert_same(got, oracle_run(boom, mode=mode, max_attempts=cap), "overflow")
        frozen = inputs.replicate_batch(inputs.isomerization(), [1.0], [0, 9], 5, 10.0, 4)
        assert_same(gpu_run(frozen, layout=layout, mode=mode), oracle_run(frozen, mode=mode), "frozen")


@pytest.mark.parametrize("layout", LAYOUTS, ids=LAYOUT_IDS)
def test_degenerate_sizes(layout):
    b = inputs.mm_batch(16)
    # no simulations
    e = inputs.Batch(b.network, b.params[:0], b.x0[:0], b.t_end, b.sample_times)
    s, st = gpu_run(e, layout=layout)
    assert s.shape == (0, 11, 4) and st.shape == (0,)
    # t_end = 0: every sample is x0, nothing fires
    z = inputs.Batch(b.network, b.params, b.x0, 0.0, np.zeros(3))
    assert_same(gpu_run(z, layout=layout), oracle_run(z), "t_end=0")
    # no sample times: only counters
    n = inputs.Batch(b.network, b.params, b.x0, 5.0, np.zeros(0))
    assert_same(gpu_run(n, layout=layout), oracle_run(n), "S=0")
    # repeated sample times
    r = inputs.Batch(b.network, b.params, b.x0, 5.0, np.array([0.0, 1.0, 1.0, 5.0, 5.0]))
    assert_same(gpu_run(r, layout=layout), oracle_run(r), "repeated T")
    # a single simulation (one busy lane in the warp)
    one = inputs.random_batch(16, 32, 1, seed=6, t_end=20.0, n_samples=5)
    assert_same(gpu_run(one, layout=layout), oracle_run(one), "n=1")


@pytest.mark.parametrize("block_warps,sims_per_warp,ctas_per_sm,reg_cap",
                         [(1, 0, 0, 0), (2, 0, 0, 0), (4, 0, 0, 0), (8, 0, 0, 0), (4, 1, 0, 0), (2, 7, 0, 0),
                          (1, 16, 0, 0), (4, 0, 1, 0), (4, 0, 0, 1), (2, 16, 0, 1), (4, 0, 1, 1)])
def test_launch_shape_does_not_change_results(block_warps, sims_per_warp, ctas_per_sm, reg_cap):
    # the register-budget build and the carve-out for fewer CTAs per SM included
    b = inputs.random_batch(32, 64, 300, seed=12, t_end=20.0, n_samples=11)
    ref = gpu_run(b, seed=3, max_attempts=100_000, layout=abi.SSA_LAYOUT_WARP)
    got = gpu_run(b, seed=3, max_attempts=100_000, layout=abi.SSA_LAYOUT_LANE, block_warps=block_warps,
                  sims_per_warp=sims_per_warp, ctas_per_sm=ctas_per_sm, reg_cap=reg_cap)
    assert_same(got, ref, f"block_warps={block_warps} sims_per_warp={sims_per_warp} ctas={ctas_per_sm} reg={reg_cap}")
    if reg_cap == 0 and ctas_per_sm == 0 and block_warps == 4:
        # the 168-register build of fast mode gives the fast-mode results of the default build
        f0 = gpu_run(b, seed=3, max_attempts=100_000, precision=abi.SSA_FAST)
        f1 = gpu_run(b, seed=3, max_attempts=100_000, precision=abi.SSA_FAST, reg_cap=1)
        assert_same(f1, f0, "fast reg_cap")


def test_sharding_by_sim_offset_is_bit_identical():
    b = inputs.random_batch(16, 32, 200, seed=8, t_end=20.0, n_samples=11)
    whole = gpu_run(b, seed=9, max_attempts=100_000)
    lo = gpu_run(b, seed=9, max_attempts=100_000, rows=np.arange(0, 120))
    hi_rows = np.arange(120, 200)
    hi = gpu_run(inputs.Batch(b.network, b.params[hi_rows], b.x0[hi_rows], b.t_end, b.sample_times),
                 seed=9, max_attempts=100_000, sim_offset=120)
    assert np.array_equal(np.concatenate([lo[0], hi[0]]), whole[0])
    assert np.array_equal(np.concatenate([lo[1], hi[1]]), whole[1])


def test_host_buffer_api_matches_device_api():
    b = inputs.random_batch(16, 32, 100, seed=3, t_end=10.0, n_samples=11)
    o = abi.ssa_default_options(max_attempts=100_000)
    hs, hst = abi.simulate_host(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=4, opts=o)
    assert_same((hs, hst), gpu_run(b, seed=4, max_attempts=100_000), "host API")
    m = abi.Model(b.network)
    j = abi.ssa_submit_batch(m, b.params, b.x0, b.t_end, b.sample_times, seed=4, opts=o)
    j.wait()
    assert j.poll() == abi.SSA_JOB_DONE
    j.release()
    m.close()


# ------------------------------------- full size, sampled against the oracle

def test_full_size_32x64_sweep_sampled():
    # the 65,536-simulation 32 x 64 sweep in the benchmark's launch shape;
    # 24 simulations spread over the batch are recomputed one by one
    b = inputs.random_batch(32, 64, 65536, seed=0)
    cap = 1 << 20
    got = gpu_run(b, seed=0, max_attempts=cap)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(65536, size=24, replace=False))
    ref = oracle_run(b, seed=0, rows=rows, max_attempts=cap)
    assert_same((got[0][rows], got[1][rows]), ref, "full-size sampled")
    s, st = got
    assert s.min() >= 0
    assert np.all(s[:, 0, :] == b.x0)
    ok = st["status"] == 0
    assert np.all(st["t_final"][ok] == b.t_end)
