"""The stored full-sweep digests are the current oracle's.

tests/golden/rand32x64_65536_seed0_digests.txt holds the oracle's results of
the 65,536-simulation random 32 x 64 sweep as block digests; the GPU test
tests/test_zy_full_batch_digest.py compares the engine's full batch with
them.  Here two blocks (one with a simulation that reaches the attempt cap,
one without) are recomputed by the oracle alone, by their global simulation
indices, so a change to the oracle that leaves the stored file stale fails on
the CPU."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1309_7695_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _digests():
    spec = importlib.util.spec_from_file_location("full_batch_digest",
                                                  os.path.join(HERE, "golden", "full_batch_digest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("block", [5, 63])
def test_stored_block_digest_is_the_oracles(block):
    g = _digests()
    s = g.SWEEP
    want = g.read_digests()
    assert len(want) == s["n_sims"] // g.BLOCK
    b = inputs.random_batch(s["n_species"], s["n_reactions"], s["n_sims"], seed=s["input_seed"])
    rows = np.arange(block * g.BLOCK, (block + 1) * g.BLOCK)
    samples, stats = oracle.simulate(b.network, b.params[rows], b.x0[rows], b.t_end, b.sample_times,
                                     seed=s["sim_seed"], opts=oracle.default_opts(max_attempts=s["max_attempts"]),
                                     sim_ids=rows)
    assert g.block_digests(samples, stats) == [want[block]]
