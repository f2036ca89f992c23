"""Stores the oracle's block digests of the 16,384-simulation random
128 x 256 sweep at t_end = 100.

The sweep: the random network of 128 species and 256 reactions (network
seed 0), 16,384 parameter sets of input seed 0 (rates log-uniform in
[1e-4, 1], initial counts uniform in {0..10^4}), t_end = 100 with 101 sample
times, simulation seed 0, epsilon = 0.03, n_c = 10 and an attempt cap of
2^20 leap attempts + SSA steps per simulation.  At these counts most
simulations fall back to exact SSA blocks for long stretches, so many reach
the cap before t_end; the cap, not the horizon, is what makes the sweep
finite, and the capped fraction is written into the file's header.

    python tests/golden/rand128x256_digest.py [threads]

runs the oracle (and nothing else) over the sweep in chunks of 1,024
simulations, appending each chunk's digest to a partial file so that an
interrupted run resumes where it stopped, and finally writes
rand128x256_16384_seed0_digests.txt beside this file.  The digest of a block
is the one defined in full_batch_digest.py (trajectories, then status and
counters)."""
from __future__ import annotations

import importlib.util
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DIGESTS = os.path.join(HERE, "rand128x256_16384_seed0_digests.txt")
PARTIAL = DIGESTS + ".partial"
SWEEP = dict(n_species=128, n_reactions=256, n_sims=16384, input_seed=0, sim_seed=0, x0_max=10_000,
             t_end=100.0, n_samples=101, max_attempts=1 << 20)


def _block_module():
    spec = importlib.util.spec_from_file_location("full_batch_digest", os.path.join(HERE, "full_batch_digest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def make_batch(inputs):
    s = SWEEP
    return inputs.random_batch(s["n_species"], s["n_reactions"], s["n_sims"], seed=s["input_seed"],
                               x0_max=s["x0_max"], t_end=s["t_end"], n_samples=s["n_samples"])


def read_digests(path=DIGESTS):
    return _block_module().read_digests(path)


def main():
    root = os.path.dirname(os.path.dirname(HERE))
    sys.path.insert(0, root)
    import oracle
    from paper_1309_7695_b300 import inputs

    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    g = _block_module()
    s = SWEEP
    b = make_batch(inputs)
    opts = oracle.default_opts(max_attempts=s["max_attempts"])
    done = {}
    if os.path.exists(PARTIAL):
        for ln in open(PARTIAL):
            f = ln.split()
            done[int(f[0])] = f[1:]
    for b0 in range(0, s["n_sims"], g.BLOCK):
        if b0 in done:
            continue
        rows = np.arange(b0, b0 + g.BLOCK)
        t0 = time.perf_counter()
        samples, stats = oracle.simulate_batch(b, seed=s["sim_seed"], opts=opts, rows=rows, threads=threads)
        (dig,) = g.block_digests(samples, stats, block=g.BLOCK)
        counts = [int((stats["status"] == k).sum()) for k in range(5)]
        tot = [int(stats[f].sum()) for f in ("firings", "leaps", "ssa_steps", "rejected")]
        with open(PARTIAL, "a") as f:
            f.write(f"{b0} {dig} {' '.join(map(str, counts))} {' '.join(map(str, tot))}\n")
        done[b0] = [dig, *map(str, counts), *map(str, tot)]
        print(f"block {b0}: {time.perf_counter() - t0:.1f} s, status counts {counts}", flush=True)
    status = np.zeros(5, dtype=np.int64)
    tot = np.zeros(4, dtype=np.int64)
    for v in done.values():
        status += np.asarray(v[1:6], dtype=np.int64)
        tot += np.asarray(v[6:10], dtype=np.int64)
    with open(DIGESTS, "w") as f:
        f.write("# Oracle results of the random 128 x 256 sweep, 16,384 simulations (input seed 0, x0 in\n"
                "# {0..10^4}, simulation seed 0, t_end 100, 101 sample times, eps 0.03, n_c 10, attempt cap\n"
                "# 2^20), as SHA-256 digests of blocks of 1,024 simulations.  Written by\n"
                "# tests/golden/rand128x256_digest.py, which calls only the oracle.\n")
        f.write(f"# firings {tot[0]}, leaps {tot[1]}, ssa_steps {tot[2]}, rejected {tot[3]}; status counts "
                f"OK {status[0]}, STEP_LIMIT {status[1]}, OVERFLOW {status[2]}, REJECT_LIMIT {status[3]}, "
                f"INVALID {status[4]}; capped fraction {status[1] / s['n_sims']:.4f}\n")
        for b0 in sorted(done):
            f.write(f"{b0} {done[b0][0]}\n")
    os.unlink(PARTIAL)
    print(f"wrote {len(done)} block digests to {DIGESTS}")


if __name__ == "__main__":
    main()
