"""Every simulation of the benchmark-size sweep equals the oracle's.

The random 32 x 64 sweep of 65,536 parameter sets (the benchmark's batch,
simulation seed 0, attempt cap 2^20) is simulated by the engine in FP64
reference mode, in the benchmark's launch shape, and its trajectories and
counters are compared with the oracle's through SHA-256 digests of blocks of
1,024 simulations.  The oracle needs minutes of CPU time for the whole batch,
so its digests were computed once by tests/golden/full_batch_digest.py (which
calls only the oracle) and stored beside it.  The file runs last because it
repeats the full-size launch."""
import importlib.util
import os

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1309_7695_b300 import inputs  # noqa: E402
from test_gpu_parity import gpu_run  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _digests():
    spec = importlib.util.spec_from_file_location("full_batch_digest",
                                                  os.path.join(HERE, "golden", "full_batch_digest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_simulation_of_the_full_sweep_equals_the_oracle():
    g = _digests()
    s = g.SWEEP
    b = inputs.random_batch(s["n_species"], s["n_reactions"], s["n_sims"], seed=s["input_seed"])
    samples, stats = gpu_run(b, seed=s["sim_seed"], max_attempts=s["max_attempts"])
    got = g.block_digests(samples, stats)
    want = g.read_digests()
    assert len(got) == len(want) == s["n_sims"] // g.BLOCK
    bad = [k * g.BLOCK for k, (a, w) in enumerate(zip(got, want)) if a != w]
    assert not bad, f"{len(bad)} blocks differ from the oracle; first simulations of the blocks: {bad[:10]}"
