"""Block digests of a simulation batch's results, and the script that stores
the oracle's digests of the 65,536-simulation random 32 x 64 sweep.

A block is 1,024 consecutive simulations.  Its digest is the SHA-256 of the
block's int32 trajectories (simulation, sample time, species; C order,
little-endian) followed by its counters: status (int32), leaps, rejected,
ssa_steps, firings, attempts (int64) and the bits of t_final (float64).
Equal digests mean bit-identical results.

    python tests/golden/full_batch_digest.py

runs the oracle (and nothing else) on the sweep that the full-size GPU test
simulates -- 32 species x 64 reactions, network seed 0, 65,536 parameter
sets of input seed 0, t_end = 100, 101 sample times, simulation seed 0,
epsilon = 0.03, n_c = 10, attempt cap 2^20 -- and writes
rand32x64_65536_seed0_digests.txt beside this file."""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

BLOCK = 1024
FIELDS = (("status", "<i4"), ("leaps", "<i8"), ("rejected", "<i8"), ("ssa_steps", "<i8"), ("firings", "<i8"),
          ("attempts", "<i8"), ("t_final", "<f8"))
HERE = os.path.dirname(os.path.abspath(__file__))
DIGESTS = os.path.join(HERE, "rand32x64_65536_seed0_digests.txt")
SWEEP = dict(n_species=32, n_reactions=64, n_sims=65536, input_seed=0, sim_seed=0, max_attempts=1 << 20)


def block_digests(samples, stats, block=BLOCK):
    """One hex SHA-256 per block of `block` simulations (see the module text)."""
    n = samples.shape[0]
    out = []
    for b0 in range(0, n, block):
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(samples[b0:b0 + block], dtype="<i4").tobytes())
        for name, dt in FIELDS:
            h.update(np.ascontiguousarray(stats[name][b0:b0 + block]).astype(dt).tobytes())
        out.append(h.hexdigest())
    return out


def read_digests(path=DIGESTS):
    return [ln.split()[1] for ln in open(path) if ln.strip() and not ln.startswith("#")]


def main():
    root = os.path.dirname(os.path.dirname(HERE))
    sys.path.insert(0, root)
    import oracle
    from paper_1309_7695_b300 import inputs

    s = SWEEP
    b = inputs.random_batch(s["n_species"], s["n_reactions"], s["n_sims"], seed=s["input_seed"])
    samples, stats = oracle.simulate(b.network, b.params, b.x0, b.t_end, b.sample_times, seed=s["sim_seed"],
                                     opts=oracle.default_opts(max_attempts=s["max_attempts"]))
    digests = block_digests(samples, stats)
    capped = int((stats["status"] == 1).sum())
    with open(DIGESTS, "w") as f:
        f.write("# Oracle results of the random 32 x 64 sweep, 65,536 simulations (input seed 0, simulation\n"
                "# seed 0, t_end 100, 101 sample times, eps 0.03, n_c 10, attempt cap 2^20), as SHA-256\n"
                "# digests of blocks of 1,024 simulations.  Written by tests/golden/full_batch_digest.py,\n"
                "# which calls only the oracle.\n")
        f.write(f"# firings {int(stats['firings'].sum())}, leaps {int(stats['leaps'].sum())}, "
                f"ssa_steps {int(stats['ssa_steps'].sum())}, capped simulations {capped}\n")
        for k, d in enumerate(digests):
            f.write(f"{k * BLOCK} {d}\n")
    print(f"wrote {len(digests)} block digests to {DIGESTS}")


if __name__ == "__main__":
    main()
