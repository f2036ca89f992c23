"""The seeded input generators follow their stated rules.

Every parity test, the benchmark and the CPU baseline draw their networks and
sweeps from ``paper_1309_7695_b300/inputs.py``; these CPU checks pin the
generator's rules (reaction-order mix, product counts, coefficient ranges,
rate and count ranges, sample-time grid, the heterogeneous group draw) and
its determinism, so that a workload named by its sizes and seed is the same
workload everywhere."""
import numpy as np
import pytest

from paper_1309_7695_b300 import inputs


@pytest.mark.parametrize("n,m,seed", [(32, 64, 0), (128, 256, 3), (4, 8, 1), (256, 512, 7), (2, 9, 5)])
def test_random_network_rules(n, m, seed):
    net = inputs.random_network(n, m, seed)
    assert net.n_species == n and net.n_reactions == m
    orders = net.orders()
    # exactly floor(M/4) order-0 and floor(M/4) order-2 reactions, the rest order 1
    assert (orders == 0).sum() == m // 4
    assert (orders == 2).sum() == m // 4
    assert (orders == 1).sum() == m - 2 * (m // 4)
    for r, p, o in zip(net.reactants, net.products, orders):
        for s, c in r + p:
            assert 0 <= s < n
        # a repeated species in an order-2 reaction is one 2X entry
        species = [s for s, _ in r]
        assert len(species) == len(set(species))
        assert all(c in (1, 2) for _, c in r)
        # products: distinct species, coefficients in {1, 2}, 1-2 of them
        # for order 0 and 0-2 otherwise (never more than N)
        ps = [s for s, _ in p]
        assert len(ps) == len(set(ps))
        assert all(c in (1, 2) for _, c in p)
        assert (1 if o == 0 else 0) <= len(p) <= min(2, n)
    # the shuffle: order-0 reactions are not all at the front (M >= 8 here)
    if m >= 8:
        assert not np.all(orders[: m // 4] == 0)


def test_random_network_product_count_mix():
    # over many reactions the product counts are uniform over their ranges
    net = inputs.random_network(256, 4096, 11)
    orders = net.orders()
    counts = np.array([len(p) for p in net.products])
    c0 = np.bincount(counts[orders == 0], minlength=3)
    assert c0[0] == 0 and abs(c0[1] - c0[2]) < 0.15 * c0.sum()
    c12 = np.bincount(counts[orders > 0], minlength=3) / (orders > 0).sum()
    assert np.all(np.abs(c12 - 1 / 3) < 0.05)
    coefs = np.array([c for p in net.products for _, c in p])
    assert abs((coefs == 1).mean() - 0.5) < 0.05
    # order 2: a repeat (2X) has probability 1/N
    two = [r for r, o in zip(net.reactants, orders) if o == 2]
    assert sum(1 for r in two if len(r) == 1) < 0.05 * len(two)


def test_random_network_is_a_function_of_its_sizes_and_seed():
    a = inputs.random_network(32, 64, 4)
    b = inputs.random_network(32, 64, 4)
    c = inputs.random_network(32, 64, 5)
    assert a.reactants == b.reactants and a.products == b.products
    assert a.reactants != c.reactants or a.products != c.products


def test_csr_and_stoichiometry_agree():
    net = inputs.random_network(16, 40, 2)
    csr = net.csr()
    nu = net.stoichiometry()
    dense = np.zeros((net.n_species, net.n_reactions), dtype=np.int64)
    for side, sign in (("react", -1), ("prod", 1)):
        ptr, sp, cf = csr[f"{side}_ptr"], csr[f"{side}_species"], csr[f"{side}_coef"]
        assert ptr[0] == 0 and ptr[-1] == len(sp) and np.all(np.diff(ptr) >= 0)
        for j in range(net.n_reactions):
            row = sp[ptr[j]:ptr[j + 1]]
            assert np.all(np.diff(row) > 0)   # sorted, one entry per species
            for s, c in zip(row, cf[ptr[j]:ptr[j + 1]]):
                dense[s, j] += sign * c
    assert np.array_equal(dense, nu)
    rp, rc = csr["react_ptr"], csr["react_coef"]
    assert net.orders().tolist() == [int(rc[rp[j]:rp[j + 1]].sum()) for j in range(net.n_reactions)]


def test_random_batch_ranges():
    b = inputs.random_batch(32, 64, 5000, seed=9)
    assert b.params.shape == (5000, 64) and b.params.dtype == np.float64
    assert b.x0.shape == (5000, 32) and b.x0.dtype == np.int32
    assert b.params.min() >= 1e-4 and b.params.max() <= 1.0
    # log-uniform: log10 of the rates is uniform on [-4, 0]
    lg = np.log10(b.params)
    assert abs(lg.mean() + 2.0) < 0.02 and abs(lg.std() - 4 / np.sqrt(12)) < 0.02
    assert b.x0.min() >= 0 and b.x0.max() <= 1000
    assert abs(b.x0.mean() - 500) < 5
    assert b.t_end == 100.0 and len(b.sample_times) == 101
    again = inputs.random_batch(32, 64, 5000, seed=9)
    assert np.array_equal(again.params, b.params) and np.array_equal(again.x0, b.x0)


@pytest.mark.parametrize("t_end,s", [(10.0, 11), (100.0, 101), (0.3, 7), (1e-3, 2), (5.0, 1), (1000.0, 200)])
def test_uniform_sample_times(t_end, s):
    T = inputs.uniform_sample_times(t_end, s)
    assert len(T) == s and T[-1] == t_end
    assert np.all(np.diff(T) > 0) and np.all(T <= t_end) and T[0] >= 0
    if s > 1:
        k = np.arange(s - 1, dtype=np.float64)
        assert np.array_equal(T[:-1], (k * t_end) / float(s - 1))
        assert T[0] == 0.0


def test_mm_batch_ranges_and_volume_scaling():
    b = inputs.mm_batch(2000, seed=1)
    assert b.network.n_species == 4 and b.network.n_reactions == 3
    assert np.all(b.x0 == [200, 500, 0, 0])
    k1, k2, k3 = b.params.T
    assert k1.min() >= 1e-3 and k1.max() <= 1e-2
    assert k2.min() >= 1e-2 and k2.max() <= 1.0 and k3.min() >= 1e-2 and k3.max() <= 1.0
    s = inputs.mm_batch(2000, seed=1, scale=10.0)
    assert np.all(s.x0 == [2000, 5000, 0, 0])
    assert np.allclose(s.params[:, 0], k1 / 10.0, rtol=0, atol=0)
    assert np.array_equal(s.params[:, 1:], b.params[:, 1:])
    assert list(b.sample_times) == [float(k) for k in range(11)]


def test_hetero_groups_draw():
    groups = inputs.hetero_groups(200_000, seed=0)
    assert sum(g.n_sims for g in groups) == 200_000
    sizes = {(g.network.n_species, g.network.n_reactions) for g in groups}
    assert sizes <= {(m // 2, m) for m in (8, 16, 32, 64, 128, 256, 384, 512)}
    assert len(sizes) == 8   # ~50 groups reach every network
    for g in groups[:-1]:
        assert 16 <= g.n_sims <= 8192
        assert 10.0 <= g.t_end <= 1000.0
        assert len(g.sample_times) == 101 and g.sample_times[-1] == g.t_end
        # one parameterization per group, replicated
        assert np.all(g.params == g.params[0]) and np.all(g.x0 == g.x0[0])
    assert 1 <= groups[-1].n_sims <= 8192   # the last group is truncated
    # groups of one network share the network object (one model load each)
    by_size = {}
    for g in groups:
        by_size.setdefault(g.network.n_reactions, set()).add(id(g.network))
    assert all(len(v) == 1 for v in by_size.values())
