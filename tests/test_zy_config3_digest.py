"""Every simulation of the 128 x 256 sweep at t_end = 100 equals the oracle's.

The random network of 128 species and 256 reactions, 16,384 parameter sets
with initial counts up to 10^4, t_end = 100 with 101 sample times, attempt
cap 2^20, is simulated by the engine in FP64 reference mode in the default
launch shape, and its trajectories and counters are compared with the
oracle's through SHA-256 digests of blocks of 1,024 simulations.  The oracle
needs about an hour of CPU time for the sweep, so its digests were computed
once by tests/golden/rand128x256_digest.py (which calls only the oracle) and
stored beside it; the file's header gives the capped fraction.  The test also
checks that the engine's capped fraction and totals equal that header."""
import importlib.util
import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import inputs  # noqa: E402
from test_gpu_parity import gpu_run  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _module(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(HERE, "golden", name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_simulation_of_the_128x256_sweep_equals_the_oracle():
    g = _module("rand128x256_digest")
    blocks = _module("full_batch_digest")
    s = g.SWEEP
    b = g.make_batch(inputs)
    samples, stats = gpu_run(b, seed=s["sim_seed"], max_attempts=s["max_attempts"])
    got = blocks.block_digests(samples, stats)
    want = g.read_digests()
    assert len(got) == len(want) == s["n_sims"] // blocks.BLOCK
    bad = [k * blocks.BLOCK for k, (a, w) in enumerate(zip(got, want)) if a != w]
    assert not bad, f"{len(bad)} blocks differ from the oracle; first simulations of the blocks: {bad[:10]}"
    header = open(g.DIGESTS).read()
    capped = int(re.search(r"STEP_LIMIT (\d+)", header).group(1))
    firings = int(re.search(r"# firings (\d+)", header).group(1))
    assert int((stats["status"] == 1).sum()) == capped
    assert int(np.asarray(stats["firings"], dtype=np.int64).sum()) == firings
