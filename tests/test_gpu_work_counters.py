"""The launch's work counters (ssa_options.work_counters) count the method's
work, not the schedule's: the same simulations give the same counts in any
launch shape, single or persistent multi-group launch, and on a replay, and
the counts obey the relations the method implies.  The benchmark relies on
this: it times a launch without counters and counts an untimed replay."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi, inputs  # noqa: E402

DEV = torch.device("cuda:0")
CAP = 100_000


def counted(batch, model, seed, precision=abi.SSA_FP64_REF, multi=False, **shape):
    n, N, S = batch.n_sims, batch.network.n_species, len(batch.sample_times)
    p = torch.from_numpy(batch.params).to(DEV)
    x = torch.from_numpy(batch.x0).to(DEV)
    T = torch.from_numpy(batch.sample_times).to(DEV)
    out = torch.empty((n, S, N), dtype=torch.int32, device=DEV)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)
    work = torch.zeros(abi.SSA_WORK_COUNTERS, dtype=torch.int64, device=DEV)
    o = abi.ssa_default_options(precision=precision, max_attempts=CAP, work_counters=work.data_ptr(), **shape)
    if multi:
        half = n // 2
        groups = [dict(model=model, params=p[:half], x0=x[:half], sample_times=T, samples=out[:half],
                       stats=st[:half], t_end=batch.t_end, seed=seed, sim_offset=0),
                  dict(model=model, params=p[half:], x0=x[half:], sample_times=T, samples=out[half:],
                       stats=st[half:], t_end=batch.t_end, seed=seed, sim_offset=half)]
        abi.ssa_simulate_multi_dev(groups[::-1], opts=o)
    else:
        abi.ssa_simulate_dev(model, p, x, batch.t_end, T, out, st, seed=seed, opts=o)
    torch.cuda.synchronize()
    return work.cpu().numpy(), st.cpu().numpy().view(abi.STATS_DTYPE).reshape(n)


@pytest.mark.parametrize("precision", [abi.SSA_FP64_REF, abi.SSA_FAST], ids=["fp64", "fast"])
def test_work_counts_do_not_depend_on_the_schedule(precision):
    b = inputs.random_batch(32, 64, 600, seed=14, t_end=30.0, n_samples=11)
    m = abi.Model(b.network)
    try:
        ref, st = counted(b, m, 9, precision)
        assert (ref > 0).all(), dict(zip(abi.WORK_NAMES, ref))
        for shape in [dict(block_warps=2), dict(block_warps=8, sims_per_warp=7), dict(reg_cap=1),
                      dict(ctas_per_sm=1)]:
            got, _ = counted(b, m, 9, precision, **shape)
            assert np.array_equal(got, ref), shape
        got, st2 = counted(b, m, 9, precision, multi=True)
        assert np.array_equal(got, ref), "persistent multi-group launch"
        assert np.array_equal(st2["firings"], st["firings"])
    finally:
        m.close()
    w = dict(zip(abi.WORK_NAMES, ref.astype(np.int64)))
    attempts = int(st["leaps"].sum() + st["rejected"].sum())
    # every leap attempt follows a step selection, forms at most M means and evaluates tau'' at most once;
    # every PTRS draw takes at least one iteration and at most one acceptance test per iteration
    assert w["selections"] >= 1 and w["tau2"] <= attempts
    assert w["means"] <= 64 * attempts and w["inv_draws"] + w["ptrs_draws"] <= w["means"]
    assert w["ptrs_iters"] >= w["ptrs_draws"] and w["ptrs_tests"] <= w["ptrs_iters"]
    assert w["tau_species"] <= 32 * w["selections"] and w["tau_terms"] >= w["tau_species"]


def test_counting_changes_no_result():
    b = inputs.random_batch(16, 32, 300, seed=15, t_end=20.0, n_samples=11)
    m = abi.Model(b.network)
    try:
        n, N, S = b.n_sims, 16, 11
        p = torch.from_numpy(b.params).to(DEV)
        x = torch.from_numpy(b.x0).to(DEV)
        T = torch.from_numpy(b.sample_times).to(DEV)
        outs = []
        for with_work in (False, True):
            out = torch.empty((n, S, N), dtype=torch.int32, device=DEV)
            work = torch.zeros(abi.SSA_WORK_COUNTERS, dtype=torch.int64, device=DEV)
            o = abi.ssa_default_options(max_attempts=CAP, work_counters=work.data_ptr() if with_work else None)
            abi.ssa_simulate_dev(m, p, x, b.t_end, T, out, None, seed=4, opts=o)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
    finally:
        m.close()
