"""The benchmark's roofline bookkeeping, on the CPU.

The roofline's `achieved` is the method's FP64 operations counted from the
launch's counters (bench.algorithmic_fp64_ops) and its `traffic` the
measured DRAM bytes per simulation times the simulations of the launch
(bench.traffic_per_launch).  These tests pin each counter's per-unit cost,
the order in which the work counters are read (it must be the library's
SSA_WORK_* order), and the scaling of the traffic with the schedule."""
import types

import numpy as np
import pytest

import bench
from paper_1309_7695_b300 import abi, inputs


def _stats(ssa=0, leaps=0, rejected=0):
    s = np.zeros(1, dtype=abi.STATS_DTYPE)
    s["ssa_steps"], s["leaps"], s["rejected"] = ssa, leaps, rejected
    return s


def test_propensity_multiplies():
    # E + S -> ES: (c x) y, two multiplies; ES -> E + S and ES -> E + P: c x, one each
    assert bench.propensity_ops(inputs.michaelis_menten()) == 4
    net = inputs.Network(2, [[], [(0, 2)], [(0, 1), (1, 1)]], [[(0, 1)], [(1, 1)], [(0, 1)]])
    assert bench.propensity_ops(net) == 0 + 1 + 2


def test_work_counter_order_is_the_librarys():
    # algorithmic_fp64_ops reads the work counters by position; the positions
    # are the SSA_WORK_* indices of include/tauleap.h
    names = ("selections", "tau_terms", "tau_species", "tau2", "means", "inv_draws", "inv_terms",
             "ptrs_draws", "ptrs_iters", "ptrs_tests")
    assert tuple(abi.WORK_NAMES[:len(names)]) == names
    assert [getattr(abi, "SSA_WORK_" + n.upper()) for n in names] == list(range(len(names)))


@pytest.mark.parametrize("counter, cost", [
    ("selections", "P + 2M + 1"), ("tau_terms", 4), ("tau_species", 5), ("tau2", 23), ("means", 1),
    ("inv_draws", 18), ("inv_terms", 3), ("ptrs_draws", 8), ("ptrs_iters", 6), ("ptrs_tests", 70)])
def test_each_work_counter_costs_what_the_model_states(counter, cost):
    net = inputs.random_network(32, 64, 0)
    P, M = bench.propensity_ops(net), net.n_reactions
    work = np.zeros(abi.SSA_WORK_COUNTERS)
    work[list(abi.WORK_NAMES).index(counter)] = 1
    want = P + 2 * M + 1 if cost == "P + 2M + 1" else cost
    assert bench.algorithmic_fp64_ops(_stats(), work, net) == want


def test_ssa_events_and_leap_attempts():
    net = inputs.random_network(32, 64, 0)
    P, M = bench.propensity_ops(net), net.n_reactions
    none = np.zeros(abi.SSA_WORK_COUNTERS)
    assert bench.algorithmic_fp64_ops(_stats(ssa=1), none, net) == P + M / 32 + 30
    # an accepted and a rejected attempt each cost the step choice and the clock
    assert bench.algorithmic_fp64_ops(_stats(leaps=3, rejected=2), none, net) == 2 * 5
    # the model is linear in every counter
    work = np.arange(1, abi.SSA_WORK_COUNTERS + 1, dtype=np.float64)
    parts = sum(bench.algorithmic_fp64_ops(_stats(), np.where(np.arange(len(work)) == k, work, 0), net)
                for k in range(len(work)))
    assert bench.algorithmic_fp64_ops(_stats(), work, net) == pytest.approx(parts, rel=1e-15)


def test_traffic_scales_with_the_simulations_of_the_launch():
    n = 65536
    per = bench.TRAFFIC_BYTES_PER_SIM
    multi = types.SimpleNamespace(layout=0, schedule="multi", steps=20)
    assert bench.traffic_per_launch(multi, "fp64", n) == per["RefArith"] * n * 20
    assert bench.traffic_per_launch(multi, "fast", n) == per["FastArith"] * n * 20
    for sched in ("serial", "streams"):
        one = types.SimpleNamespace(layout=0, schedule=sched, steps=20)
        assert bench.traffic_per_launch(one, "fp64", n) == per["RefArith"] * n
    warp = types.SimpleNamespace(layout=1, schedule="multi", steps=20)
    assert bench.traffic_per_launch(warp, "fp64", n) is None
    # the measured bytes lie just above the algorithmic bytes of the 32 x 64
    # workload: 8M + 4N read, 4 N S + 56 written per simulation
    algorithmic = 8 * 64 + 4 * 32 + 4 * 32 * 101 + 56
    for v in per.values():
        assert algorithmic < v < 1.1 * algorithmic


def test_ordinals():
    assert [bench.ordinal(k) for k in (1, 2, 3, 4, 11, 12, 13, 21, 22, 32, 101, 111, 256)] == \
        ["1st", "2nd", "3rd", "4th", "11th", "12th", "13th", "21st", "22nd", "32nd", "101st", "111th", "256th"]
