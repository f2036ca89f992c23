"""The multi-rank path on the CPU: world_size 2 over gloo.

Each rank simulates its shard of a small sweep with the oracle (standing in
for the engine, which needs a GPU) at its global simulation offset; the
gathered shards must equal the unsharded run bit for bit, and the
end-of-run reduction must return the slowest rank's time and the summed
counters."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1309_7695_b300 import inputs, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = inputs.random_batch(16, 32, 45, seed=13, t_end=10.0, n_samples=6)
        lo, hi = shard.shard_range(rank, world, b.n_sims)
        o = oracle.default_opts(max_attempts=50_000)
        s, st = oracle.simulate(b.network, b.params[lo:hi], b.x0[lo:hi], b.t_end, b.sample_times, seed=3, opts=o,
                                sim_offset=lo)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, s, st))
        t, c = shard.reduce_run(1.0 + rank, [float(st["firings"].sum()), float(hi - lo)])
        if rank == 0:
            np.savez(os.path.join(out_dir, "shards.npz"),
                     samples=np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])]),
                     stats=np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])]),
                     t=t, c=np.array(c))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_exactly():
    from paper_1309_7695_b300 import shard

    for n in (0, 1, 7, 45, 65536):
        for w in (1, 2, 3, 8):
            r = [shard.shard_range(k, w, n) for k in range(w)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    assert shard.weak_offset(3, 65536) == 3 * 65536
    with pytest.raises(ValueError):
        shard.shard_range(2, 2, 10)


def test_two_gloo_ranks_equal_the_unsharded_run(tmp_path):
    import oracle
    from paper_1309_7695_b300 import inputs

    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "shards.npz")
    b = inputs.random_batch(16, 32, 45, seed=13, t_end=10.0, n_samples=6)
    s, st = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=3,
                            opts=oracle.default_opts(max_attempts=50_000))
    assert np.array_equal(got["samples"], s)
    assert np.array_equal(got["stats"], st)
    assert float(got["t"]) == 2.0                       # the slower rank
    assert got["c"][0] == float(st["firings"].sum())    # summed counters
    assert got["c"][1] == 45.0
