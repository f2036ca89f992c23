"""Continuous-batching server (ssa_server_*): results are the same alone and
in a mix, admission respects the HBM budget, oversized requests are
refused, and FP64 requests equal the oracle."""
import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import abi  # noqa: E402


def requests():
    nets = [inputs.random_network(8, 16, 3), inputs.random_network(24, 48, 4), inputs.michaelis_menten()]
    rng = np.random.default_rng(9)
    reqs = []
    for k in range(9):
        net = nets[k % 3]
        n = int(rng.integers(1, 400))
        t_end = float(rng.uniform(1.0, 20.0))
        S = int(rng.integers(2, 30))
        params = inputs.log_uniform(rng, 1e-3, 1.0, (n, net.n_reactions))
        x0 = rng.integers(0, 300, size=(n, net.n_species)).astype(np.int32)
        reqs.append((net, params, x0, t_end, inputs.uniform_sample_times(t_end, S), 1000 + k))
    return nets, reqs


def run_alone(server, models, reqs):
    out = []
    for net, p, x, t_end, T, seed in reqs:
        t = server.submit(models[net.name], p, x, t_end, T, seed)
        out.append(server.fetch(t))
    return out


def test_same_alone_and_in_the_mix():
    nets, reqs = requests()
    models = {n.name: abi.Model(n) for n in nets}
    opts = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=200_000)
    srv = abi.Server(n_streams=4, max_batch=4, opts=opts)
    alone = run_alone(srv, models, reqs)
    tickets = [srv.submit(models[net.name], p, x, t_end, T, seed) for net, p, x, t_end, T, seed in reqs]
    infos = [srv.wait(t) for t in tickets]
    mixed = [srv.fetch(t) for t in tickets]
    for (a, ast), (m, mst) in zip(alone, mixed):
        assert np.array_equal(a, m)
        assert np.array_equal(ast, mst)
    assert max(i.batch_size for i in infos) > 1            # requests were batched together
    for i in infos:
        assert i.state == abi.SSA_JOB_DONE and 0 <= i.t_submit <= i.t_admit <= i.t_done
    assert srv.stats()["device_bytes_in_use"] == 0
    srv.close()


def test_admission_under_a_small_budget():
    nets, reqs = requests()
    models = {n.name: abi.Model(n) for n in nets}
    opts = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=200_000)
    ref_srv = abi.Server(opts=opts)
    alone = run_alone(ref_srv, models, reqs)
    ref_srv.close()
    footprint = [p.nbytes + x.nbytes + T.nbytes + 4 * p.shape[0] * len(T) * net.n_species + 56 * p.shape[0] + 2560
                 for net, p, x, t_end, T, seed in reqs]
    srv = abi.Server(max_device_bytes=max(footprint) + 1024, n_streams=4, opts=opts)
    tickets = [srv.submit(models[net.name], p, x, t_end, T, seed) for net, p, x, t_end, T, seed in reqs]
    got = []
    for t in tickets:               # fetching releases memory and lets the queue move
        got.append(srv.fetch(t))
    for (a, ast), (g, gst) in zip(alone, got):
        assert np.array_equal(a, g) and np.array_equal(ast, gst)
    with pytest.raises(abi.SsaError) as e:
        net, p, x, t_end, T, seed = reqs[0]
        big = np.repeat(p, 5000, axis=0)
        srv.submit(models[net.name], big, np.repeat(x, 5000, axis=0), t_end, T, seed)
    assert e.value.code == abi.SSA_ENOMEM
    srv.close()


def test_fp64_requests_equal_the_oracle():
    nets, reqs = requests()
    models = {n.name: abi.Model(n) for n in nets}
    opts = abi.ssa_default_options(precision=abi.SSA_FP64_REF, max_attempts=200_000)
    srv = abi.Server(opts=opts)
    tickets = [srv.submit(models[net.name], p, x, t_end, T, seed) for net, p, x, t_end, T, seed in reqs[:5]]
    for t, (net, p, x, t_end, T, seed) in zip(tickets, reqs[:5]):
        s, st = srv.fetch(t)
        rs, rst = oracle.simulate(net, p, x, t_end, T, seed=seed, opts=oracle.default_opts(max_attempts=200_000))
        assert np.array_equal(s, rs)
        assert np.array_equal(st["firings"], rst["firings"])
    srv.close()


def test_short_request_completes_before_the_long_one_it_is_batched_with():
    # one stream slot: while a first request runs, a long and a short request
    # queue up and are then admitted together into one launch; the short one
    # must complete (and be fetchable) long before the launch ends
    long_b = inputs.random_batch(32, 64, 2048, seed=3, t_end=100.0, n_samples=11)
    short_b = inputs.mm_batch(8, seed=4, t_end=1.0, n_samples=3)
    models = {b.network.name: abi.Model(b.network) for b in (long_b, short_b)}
    opts = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=1 << 18)
    srv = abi.Server(n_streams=1, max_batch=4, opts=opts)

    def submit(b, seed):
        return srv.submit(models[b.network.name], b.params, b.x0, b.t_end, b.sample_times, seed)

    first = submit(long_b, 1)
    t_long, t_short = submit(long_b, 2), submit(short_b, 3)
    s_short, st_short = srv.fetch(t_short)
    i_long = srv.poll(t_long)
    assert i_long.t_done < 0, "the long request should still be running when the short one is fetched"
    i_long = srv.wait(t_long)
    srv.fetch(t_long)
    srv.fetch(first)
    alone = run_alone(srv, models, [(short_b.network, short_b.params, short_b.x0, short_b.t_end,
                                     short_b.sample_times, 3)])
    assert np.array_equal(alone[0][0], s_short) and np.array_equal(alone[0][1], st_short)
    assert i_long.batch_size == 2
    srv.close()
