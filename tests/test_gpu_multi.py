"""The multi-network persistent launch (ssa_simulate_multi_dev).

In FP64 reference mode every group's results equal, bit for bit, both a
single-network launch of that group and the CPU oracle, whatever the order
of the groups in the launch (a simulation's random stream depends only on
its seed and global index)."""
import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402

DEV = torch.device("cuda:0")
CAP = 100_000


def groups_fixture():
    return [
        (inputs.mm_batch(300, seed=5), 11),
        (inputs.random_batch(16, 32, 250, seed=6, t_end=20.0, n_samples=11), 12),
        (inputs.random_batch(32, 64, 150, seed=7, t_end=10.0, n_samples=6), 13),
        (inputs.replicate_batch(inputs.birth_death(), [10.0, 0.1], [0], 77, 30.0, 4), 14),
        (inputs.random_batch(40, 33, 90, seed=8, t_end=15.0, n_samples=9), 15),
    ]


def to_dev(batch, model, seed):
    n, N, S = batch.n_sims, batch.network.n_species, len(batch.sample_times)
    return {"model": model, "params": torch.from_numpy(batch.params).to(DEV),
            "x0": torch.from_numpy(batch.x0).to(DEV), "sample_times": torch.from_numpy(batch.sample_times).to(DEV),
            "samples": torch.full((n, S, N), -3, dtype=torch.int32, device=DEV),
            "stats": torch.zeros((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV),
            "t_end": batch.t_end, "seed": seed}


def fetch(g):
    n = g["params"].shape[0]
    return g["samples"].cpu().numpy(), g["stats"].cpu().numpy().view(abi.STATS_DTYPE).reshape(n)


@pytest.mark.parametrize("order,reg_cap", [([0, 1, 2, 3, 4], 0), ([4, 2, 0, 3, 1], 0), ([4, 2, 0, 3, 1], 1)],
                         ids=["given", "shuffled", "shuffled-168reg"])
@pytest.mark.parametrize("mode", [abi.SSA_MODE_TAU_LEAP, abi.SSA_MODE_EXACT], ids=["tau", "exact"])
def test_multi_equals_single_and_oracle(order, reg_cap, mode):
    fx = groups_fixture()
    models = [abi.Model(b.network) for b, _ in fx]
    opts = abi.ssa_default_options(mode=mode, max_attempts=CAP)
    multi = [to_dev(b, m, seed) for (b, seed), m in zip(fx, models)]
    abi.ssa_simulate_multi_dev([multi[k] for k in order], opts=abi.ssa_default_options(mode=mode, max_attempts=CAP,
                                                                                          reg_cap=reg_cap))
    torch.cuda.synchronize()
    for (b, seed), m, g in zip(fx, models, multi):
        single = to_dev(b, m, seed)
        abi.ssa_simulate_dev(m, single["params"], single["x0"], b.t_end, single["sample_times"], single["samples"],
                             single["stats"], seed=seed, opts=opts)
        torch.cuda.synchronize()
        ms, mst = fetch(g)
        ss, sst = fetch(single)
        assert np.array_equal(ms, ss), b.network.name
        assert np.array_equal(mst, sst), b.network.name
        rs, rst = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=seed,
                                  opts=oracle.default_opts(mode=mode, max_attempts=CAP))
        assert np.array_equal(ms, rs), b.network.name
        for f in ("status", "leaps", "rejected", "ssa_steps", "firings", "attempts"):
            assert np.array_equal(mst[f], rst[f]), (b.network.name, f)
    for m in models:
        m.close()


def test_multi_fast_mode_is_coupled_to_single_launches():
    fx = groups_fixture()
    models = [abi.Model(b.network) for b, _ in fx]
    opts = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=CAP)
    multi = [to_dev(b, m, seed) for (b, seed), m in zip(fx, models)]
    abi.ssa_simulate_multi_dev(multi, opts=opts)
    torch.cuda.synchronize()
    for (b, seed), m, g in zip(fx, models, multi):
        single = to_dev(b, m, seed)
        abi.ssa_simulate_dev(m, single["params"], single["x0"], b.t_end, single["sample_times"], single["samples"],
                             single["stats"], seed=seed, opts=opts)
        torch.cuda.synchronize()
        ms, _ = fetch(g)
        ss, _ = fetch(single)
        assert ms.min() >= 0 and np.all(ms[:, 0, :] == b.x0)
        same = np.mean((ms == ss).all(axis=(1, 2)))
        assert same > 0.9, (b.network.name, same)
    for m in models:
        m.close()


def test_multi_rejects_bad_groups():
    b = inputs.mm_batch(4)
    m = abi.Model(b.network)
    g = to_dev(b, m, 1)
    with pytest.raises(abi.SsaError):
        abi.ssa_simulate_multi_dev([g], opts=abi.ssa_default_options(layout=abi.SSA_LAYOUT_WARP))
    abi.ssa_simulate_multi_dev([], opts=None)
    m.close()
