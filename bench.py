#!/usr/bin/env python
"""Throughput benchmark of the batched tau-leaping engine.

Workload (default): one random mass-action network of 32 species and 64
reactions (orders 0/1/2 in ratio 1:2:1), 65,536 parameterizations with rate
constants log-uniform in [1e-4, 1] and initial counts uniform in {0..1000},
t_end = 100 with 101 sample times, epsilon = 0.03, n_c = 10, FP64 reference
mode (bit-exact with the CPU oracle).  Every simulation runs to t_end or to a
budget of 2^20 leap attempts + SSA steps.

A step simulates one such batch with its own seed (inputs resident in
HBM).  By default the K timed steps run as one persistent launch over the K
batches (--schedule multi): lanes take simulations from every batch through
one work counter, so a lane whose simulation ends early takes the next one
instead of idling while the long simulations of its batch finish;
--schedule streams runs one launch per batch on its own stream, and
--schedule serial one launch per batch, one after another.  Reported: reaction
firings/s (value) and sim-steps/s (accepted leaps + SSA events), the same
batches in fast mode, the same metric end to end through the host-buffer
C ABI with one job per step in flight (e2e), the roofline position of the
simulation kernel against the FP64 issue rate, and the CPU oracle on a
bounded sample of the same workload (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Other workloads (--workload): rand128x256 (the 128 x 256 sweep, 16,384
parameter sets to t_end = 100, FP64 and fast mode), hetero (uneven groups of
8 networks in one autotuned persistent launch against one launch per
network), served (a Poisson request stream through the server), rre (batched
rate-equation integration) and cle (the Langevin leap).
Multi-GPU (torchrun, one rank per GPU): each rank simulates its own 65,536
simulations (global indices rank*65536 + r), so per-GPU work is fixed
(weak scaling) and no collective is needed on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1309_7695_b300 import inputs  # noqa: E402

METRIC = "reaction firings/s & sim-steps/s (KS-matched) vs plain FP64; serve p50/p99"
WORKLOAD = dict(n_species=32, n_reactions=64, n_sims=65536, t_end=100.0, n_samples=101,
                x0_max=1000, eps=0.03, n_c=10, max_attempts=1 << 20, network_seed=0)
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes per simulation of the persistent lane kernels: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu-captured launch of 65,536 simulations of the
# workload above at an attempt cap of 2^16, divided by 65,536.  The bytes are the
# inputs read and the samples written, so they scale with the simulations a launch
# runs and not with its attempts.
TRAFFIC_BYTES_PER_SIM = {"RefArith": 14291.1, "FastArith": 14339.2}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of 65,536 simulations "
                  "(attempt cap 2^16), scaled by the simulations of this launch")
def kernel_name(args):
    """The simulation kernel a headline launch runs."""
    if args.layout == 1:
        return "warp_f64_kernel"
    arith = "RefArith" if args.precision == "fp64" else "FastArith"
    return f"lane_kernel<{arith}, {'true' if args.schedule == 'multi' else 'false'}>"


def ordinal(k):
    """1st, 2nd, 3rd, 4th, ..., 32nd: for the sample descriptions."""
    if 10 <= k % 100 <= 20:
        return f"{k}th"
    return f"{k}" + {1: "st", 2: "nd", 3: "rd"}.get(k % 10, "th")


def traffic_per_launch(args, precision, n_sims):
    """DRAM bytes of one headline launch of the lane kernel (None for the warp layout, which
    has no capture): the measured bytes per simulation times the simulations it runs."""
    if args.layout == 1:
        return None
    per_launch = n_sims * (args.steps if args.schedule == "multi" else 1)
    return TRAFFIC_BYTES_PER_SIM["RefArith" if precision == "fp64" else "FastArith"] * per_launch


def propensity_ops(net):
    """FP64 multiplies of one evaluation of all M propensities: c (order 0),
    c*x (X), (c*x)*y (X+Y), c*h (2X)."""
    ops = 0
    for row in net.reactants:
        order = sum(c for _, c in row)
        ops += 0 if order == 0 else (2 if len(row) == 2 else 1)
    return ops


def algorithmic_fp64_ops(stats, work, net):
    """FP64 operations of the method (CGP 2006 tau-leaping with the CGP 2005
    critical set and exact-SSA blocks), from the launch's counters.

    Counters: ssa_steps and leap attempts (leaps + rejected) from the
    per-simulation stats; the rest from ssa_options.work_counters.  Per unit:
      SSA event: the M propensities (P multiplies) and the O(M) selection
        (M/32 + 5 adds/compares), -ln u (22), tau = E/a0 (1), the clock (1)
        and the target u a0 (1): P + M/32 + 30;
      step selection: propensities P, the a0 and a0c sums (2M), the
        fallback threshold a0 division (1);
      tau' term (one reaction's contribution to mu_i and sigma_i^2): 2
        products and 2 adds; tau' species: eps x / g and the clamp (2), two
        divisions and bound^2 (3);
      leap attempt: the step choice and clock (2); tau'' evaluation: -ln u
        and the division (23); Poisson mean a_j tau: 1;
      inversion draw: e^-lam (17) + the first term (1), 3 per further term;
      PTRS draw: sqrt and the constants b, a, v_r (8); iteration: the
        candidate (2a/us + b) U + lam + 0.43 and the squeeze (6); acceptance
        test: two logarithms and ln k! (~70).
    Langevin increments are not counted (tau-leap mode has none)."""
    M = net.n_reactions
    P = propensity_ops(net)
    ssa = float(stats["ssa_steps"].sum())
    attempts = float(stats["leaps"].sum() + stats["rejected"].sum())
    w = {name: float(work[k]) for k, name in enumerate(
        ("selections", "tau_terms", "tau_species", "tau2", "means", "inv_draws", "inv_terms", "ptrs_draws",
         "ptrs_iters", "ptrs_tests"))}
    return (ssa * (P + M / 32 + 30) + w["selections"] * (P + 2 * M + 1) + 4 * w["tau_terms"]
            + 5 * w["tau_species"] + 2 * attempts + 23 * w["tau2"] + w["means"] + 18 * w["inv_draws"]
            + 3 * w["inv_terms"] + 8 * w["ptrs_draws"] + 6 * w["ptrs_iters"] + 70 * w["ptrs_tests"])


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_batch(rank=0):
    w = WORKLOAD
    return inputs.random_batch(w["n_species"], w["n_reactions"], w["n_sims"], seed=rank,
                               x0_max=w["x0_max"], t_end=w["t_end"], n_samples=w["n_samples"],
                               network_seed=w["network_seed"])


def config_dict(extra=None):
    w = WORKLOAD
    d = {"workload": f"random mass-action network {w['n_species']} species x {w['n_reactions']} reactions, "
                     f"{w['n_sims']} parameterizations, t_end={w['t_end']:g}, {w['n_samples']} sample times",
         "n_species": w["n_species"], "n_reactions": w["n_reactions"], "n_sims_per_gpu": w["n_sims"],
         "t_end": w["t_end"], "n_samples": w["n_samples"], "eps": w["eps"], "n_c": w["n_c"],
         "max_attempts": w["max_attempts"], "mode": "tau-leap (CGP) + SSA fallback", "precision": "fp64-ref"}
    if extra:
        d.update(extra)
    return d


def cpu_oracle_rate(batch, n_sample=2048, seed=1000, gpu_stats=None):
    """Oracle firings/s and sim-steps/s on an evenly strided sample of the
    batch (every (n/n_sample)-th simulation, so heavy and light simulations
    appear in their batch proportions), all host cores, OpenMP over
    simulations.  Rates are sample firings (steps) over sample wall time.
    ``one_core`` times an eighth of that sample on one core and again on all
    cores (firings per simulation are heavy-tailed, so only the same
    simulations compare)."""
    import oracle

    o = oracle.default_opts(eps=WORKLOAD["eps"], n_c=WORKLOAD["n_c"], max_attempts=WORKLOAD["max_attempts"])
    cores = oracle.num_threads()
    stride = max(1, batch.n_sims // n_sample)
    rows = np.arange(0, batch.n_sims, stride)

    def timed(rs, threads):
        t0 = time.perf_counter()
        _, st = oracle.simulate_batch(batch, seed=seed, opts=o, rows=rs, threads=threads)
        dt = time.perf_counter() - t0
        return float(st["firings"].sum()) / dt, float(st["leaps"].sum() + st["ssa_steps"].sum()) / dt, dt

    fir, steps, dt = timed(rows, cores)
    mix = None
    heavy = None
    if gpu_stats is not None:
        # the sample's work mix against the batch's (the GPU ran the same batch and seed), and the
        # oracle's rate on the batch's heaviest simulations, which set the length of a GPU launch
        capped = gpu_stats["status"] == 1
        att = gpu_stats["attempts"].astype(np.float64)
        mix = {"sample_capped": int(capped[rows].sum()), "batch_capped": int(capped.sum()),
               "batch_attempt_share_of_capped": float(att[capped].sum() / att.sum()),
               "sample_attempt_share_of_batch": float(att[rows].sum() / att.sum())}
        top = np.argsort(-att)[:4]
        hf, hs, hd = timed(np.sort(top), min(cores, 4))
        heavy = {"value": hf, "unit": "firings/s", "sim_steps_per_s": hs, "seconds": round(hd, 2),
                 "threads": min(cores, 4), "sample": "the 4 simulations of the batch with the most attempts "
                                                     "(one thread each)"}
    rows1 = rows[::8]
    f1, s1, d1 = timed(rows1, 1)
    fa, sa, da = timed(rows1, cores)   # the same simulations on all cores (restores the thread count)
    one_core = {"value": f1, "unit": "firings/s", "sim_steps_per_s": s1, "cores": 1, "seconds": round(d1, 2),
                "all_cores_same_sample": fa, "speedup_all_cores": d1 / da,
                "sample": f"every {ordinal(stride * 8)} simulation ({len(rows1)} simulations)"}
    return {"value": fir, "unit": "firings/s", "sim_steps_per_s": steps,
            "cores": cores, "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"every {ordinal(stride)} of the {batch.n_sims} simulations ({len(rows)} simulations, "
                      f"seed {seed}), OpenMP over simulations", "one_core": one_core, "mix": mix,
            "heaviest": heavy}


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    batch = make_batch(0)
    o = oracle.default_opts(eps=WORKLOAD["eps"], n_c=WORKLOAD["n_c"], max_attempts=WORKLOAD["max_attempts"])
    per_step = 2048   # the same sample as cpu_baseline: every 32nd simulation of the batch
    stride = batch.n_sims // per_step
    rows = np.arange(0, batch.n_sims, stride)[:per_step]
    for w in range(args.warmup):
        oracle.simulate_batch(batch, seed=2000 + w, opts=o, rows=rows)
    fir = steps = 0.0
    t0 = time.perf_counter()
    for k in range(args.steps):
        _, st = oracle.simulate_batch(batch, seed=1000 + k, opts=o, rows=rows)
        fir += float(st["firings"].sum())
        steps += float(st["leaps"].sum() + st["ssa_steps"].sum())
    dt = time.perf_counter() - t0
    value = fir / dt
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "firings/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random network and sweep)", "sim_steps_per_s": steps / dt,
            "config": config_dict({"reference_sample": f"{per_step} simulations per step (every {ordinal(stride)})"}),
            "cpu_baseline": {"value": value, "unit": "firings/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"every {ordinal(stride)} of {batch.n_sims} simulations ({per_step}) per step"},
            "e2e": {"value": value, "unit": "firings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_hetero(args):
    """Heterogeneous batch (8 networks of 8..512 reactions, log-uniform
    replicates and horizons, fast mode): one launch per network on one
    stream against one autotuned persistent multi-network launch."""
    import torch

    from paper_1309_7695_b300 import abi, autotune

    dev = torch.device("cuda:0")
    groups = inputs.hetero_groups(args.hetero_sims, seed=0)
    models, gd = {}, []
    for k, b in enumerate(groups):
        if b.network.name not in models:
            models[b.network.name] = abi.Model(b.network)
        n, N, S = b.n_sims, b.network.n_species, len(b.sample_times)
        gd.append({"model": models[b.network.name], "params": torch.from_numpy(b.params).to(dev),
                   "x0": torch.from_numpy(b.x0).to(dev), "sample_times": torch.from_numpy(b.sample_times).to(dev),
                   "samples": torch.empty((n, S, N), dtype=torch.int32, device=dev),
                   "stats": torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev),
                   "t_end": b.t_end, "seed": 100 + k})
    cap = WORKLOAD["max_attempts"]

    def totals():
        f = st = 0.0
        for g in gd:
            s = g["stats"].cpu().numpy().view(abi.STATS_DTYPE)
            f += float(s["firings"].sum())
            st += float(s["leaps"].sum() + s["ssa_steps"].sum())
        return f, st

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    o = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=cap)

    def plain():
        for g in gd:
            abi.ssa_simulate_dev(g["model"], g["params"], g["x0"], g["t_end"], g["sample_times"], g["samples"],
                                 g["stats"], seed=g["seed"], opts=o)

    t0 = time.perf_counter()
    ordered, topts, costs = autotune.plan(gd, precision=abi.SSA_FAST)
    t_plan = time.perf_counter() - t0
    topts.max_attempts = cap
    t_plain = f_plain = s_plain = None
    if not args.hetero_no_plain:
        t_plain = timed(plain)
        f_plain, s_plain = totals()
    t_multi = timed(lambda: abi.ssa_simulate_multi_dev(ordered, opts=topts))
    f_multi, s_multi = totals()
    line = {"metric": METRIC, "workload": "hetero", "value": f_multi / t_multi, "unit": "firings/s",
            "sim_steps_per_s": s_multi / t_multi, "plain_value": f_plain / t_plain if t_plain else None,
            "plain_sim_steps_per_s": s_plain / t_plain if t_plain else None,
            "speedup_vs_plain": t_plain / t_multi if t_plain else None,
            "seconds_persistent": t_multi, "seconds_plain": t_plain, "seconds_planning": t_plan,
            "dtype": "f32 propensities/Poisson, f64 clock/a0/tau'", "data": "synthetic",
            "config": {"workload": f"heterogeneous batch: {len(gd)} groups over 8 random networks (8..512 reactions, "
                                   f"species = reactions/2), replicates logU[16,8192], t_end logU[10,1000], 101 samples",
                       "n_sims": sum(int(g['params'].shape[0]) for g in gd), "max_attempts": cap,
                       "schedule": f"autotuned: most expensive group first, block_warps={topts.block_warps}, "
                                   f"sims_per_warp={topts.sims_per_warp}, reg_cap={topts.reg_cap}"}}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep128(args):
    """The 128 x 256 sweep at its full size and horizon: 16,384 parameter
    sets (initial counts up to 10^4), t_end = 100, 101 sample times, attempt
    cap 2^20, one launch in FP64 reference mode (the launch the digest test
    compares with the oracle) and one in fast mode, L2 flushed before each."""
    import torch

    from paper_1309_7695_b300 import abi

    dev = torch.device("cuda:0")
    cap = 1 << 20
    b = inputs.random_batch(128, 256, 16384, seed=0, x0_max=10_000, t_end=100.0, n_samples=101)
    n, N, S = b.n_sims, b.network.n_species, len(b.sample_times)
    model = abi.Model(b.network)
    p = torch.from_numpy(b.params).to(dev)
    x = torch.from_numpy(b.x0).to(dev)
    T = torch.from_numpy(b.sample_times).to(dev)
    out = torch.empty((n, S, N), dtype=torch.int32, device=dev)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    legs = {}
    for name, prec in (("fp64", abi.SSA_FP64_REF), ("fast", abi.SSA_FAST)):
        o = abi.ssa_default_options(precision=prec, max_attempts=cap)
        flush.fill_(7)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        abi.ssa_simulate_dev(model, p, x, b.t_end, T, out, st, seed=0, opts=o)
        e1.record()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        s = st.cpu().numpy().view(abi.STATS_DTYPE).reshape(n)
        fir = float(s["firings"].astype(np.float64).sum())
        steps = float(s["leaps"].astype(np.float64).sum() + s["ssa_steps"].astype(np.float64).sum())
        legs[name] = {"seconds": dt, "firings_per_s": fir / dt, "sim_steps_per_s": steps / dt,
                      "firings": fir, "capped_fraction": float((s["status"] == abi.SSA_STATUS_STEP_LIMIT).mean()),
                      "ssa_step_fraction": float(s["ssa_steps"].astype(np.float64).sum()) / steps}
    model.close()
    line = {"metric": METRIC, "workload": "rand128x256", "value": legs["fast"]["firings_per_s"], "unit": "firings/s",
            "sim_steps_per_s": legs["fast"]["sim_steps_per_s"], "fp64": legs["fp64"], "fast": legs["fast"],
            "fast_vs_fp64": legs["fast"]["firings_per_s"] / legs["fp64"]["firings_per_s"],
            "dtype": "f32 propensities/Poisson, f64 clock/a0/tau'", "data": "synthetic",
            "config": {"workload": "random 128 x 256 network (orders 0/1/2 in 1:2:1), 16,384 parameter sets, "
                                   "x0 U-int[0,10^4], t_end=100, 101 sample times, eps=0.03, n_c=10",
                       "max_attempts": cap, "schedule": "one launch per mode, default shape, L2 flushed before each"}}
    print(json.dumps(line), flush=True)
    return 0


def served_stream(rates, n_requests, n_networks, cap, seed=7, n_streams=4, max_batch=16):
    """Served request stream (continuous batching through abi.Server): a pool
    of random networks (M logU-int[8,512], N U-int[4,min(256,2M)]); per
    request a network from the pool, replicates logU-int[1,4096], t_end
    logU[1,500], S U-int[10,200] sample times, rates logU[1e-4,1], x0
    U{0..1000}; Poisson arrivals at each rate.  Fast mode.  Returns one dict
    per rate: p50/p99/mean latency (submit to completion), firings/s and
    sim-steps/s over the rate's wall time, launches and mean batch size."""
    import torch  # noqa: F401  (initialises the CUDA context used by the server)

    from paper_1309_7695_b300 import abi

    rng = np.random.default_rng(seed)
    pool = []
    for k in range(n_networks):
        m = int(np.floor(np.exp(rng.uniform(np.log(8), np.log(513)))))
        n = int(rng.integers(4, min(256, 2 * m) + 1))
        net = inputs.random_network(n, m, 500 + k)
        pool.append((net, abi.Model(net)))
    opts = abi.ssa_default_options(precision=abi.SSA_FAST, max_attempts=cap)
    results = []
    for lam in rates:
        srv = abi.Server(n_streams=n_streams, max_batch=max_batch, opts=opts)
        reqs = []
        for r in range(n_requests):
            net, model = pool[int(rng.integers(len(pool)))]
            reps = int(np.floor(np.exp(rng.uniform(0.0, np.log(4097)))))
            t_end = float(np.exp(rng.uniform(0.0, np.log(500.0))))
            S = int(rng.integers(10, 201))
            params = inputs.log_uniform(rng, 1e-4, 1.0, (reps, net.n_reactions))
            x0 = rng.integers(0, 1001, size=(reps, net.n_species)).astype(np.int32)
            reqs.append((model, params, x0, t_end, inputs.uniform_sample_times(t_end, S), 10_000 + r))
        gaps = rng.exponential(1.0 / lam, size=len(reqs))
        t_start = time.perf_counter()
        tickets, next_t = [], 0.0
        for (model, params, x0, t_end, T, sd), gap in zip(reqs, gaps):
            next_t += gap
            delay = next_t - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(model, params, x0, t_end, T, sd))
        lat, fir, steps, bsz = [], 0.0, 0.0, []
        for t in tickets:
            info = srv.wait(t)
            _, st = srv.fetch(t)
            lat.append(info.t_done - info.t_submit)
            bsz.append(info.batch_size)
            fir += float(st["firings"].sum())
            steps += float(st["leaps"].sum() + st["ssa_steps"].sum())
        wall = time.perf_counter() - t_start
        launches = srv.stats()["launches"]
        srv.close()
        lat = np.asarray(lat)
        results.append({"lambda_per_s": lam, "requests": len(reqs), "p50_s": float(np.percentile(lat, 50)),
                        "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                        "firings_per_s": fir / wall, "sim_steps_per_s": steps / wall, "wall_s": wall,
                        "requests_per_s": len(reqs) / wall, "launches": launches, "mean_batch": float(np.mean(bsz))})
    for _, model in pool:
        model.close()
    return results


def served_config(n_requests, n_networks, cap):
    return {"workload": f"served stream: Poisson arrivals, {n_requests} requests per rate, pool of {n_networks} random "
                        f"networks (M logU-int[8,512], N U-int[4,min(256,2M)]), replicates logU-int[1,4096], "
                        f"t_end logU[1,500], S U-int[10,200]", "max_attempts": cap,
            "server": "4 stream slots, 16 per batch, per-request completion"}


def run_served(args):
    """Served request stream: Poisson arrivals, continuous batching, p50/p99."""
    results = []
    for lam in args.serve_rates:
        results += served_stream([lam], args.serve_requests, args.serve_networks, args.serve_cap)
        print(json.dumps({"served": results[-1]}), flush=True)
    line = {"metric": METRIC, "workload": "served", "value": results[0]["p99_s"], "unit": "s (p99 latency)",
            "higher_is_better": False, "dtype": "f32 propensities/Poisson, f64 clock/a0/tau'", "data": "synthetic",
            "rates": results, "config": served_config(args.serve_requests, args.serve_networks, args.serve_cap)}
    print(json.dumps(line), flush=True)
    return 0


def rre_fp64_ops_per_attempt(net):
    """FP64 operations of one Dormand-Prince 5(4) attempt of one system.

    Six right-hand sides (the seventh stage is the next step's first): the
    mass-action rates (0 ops for order 0, 1 for X, 2 for X+Y, 3 for 2X) and,
    per net-change entry, one product and one sum; the stage combinations
    (3 + 5 + 7 + 9 + 11 ops per species, and 11 for the solution) and the
    error norm (~20 per species, one division among them)."""
    rate_ops = sum(0 if not r else (1 if len(r) == 1 and r[0][1] == 1 else (2 if len(r) == 2 else 3))
                   for r in net.reactants)
    nnz = int((net.stoichiometry() != 0).sum())
    return 6 * (rate_ops + 2 * nnz) + 66 * net.n_species


def _timed_launches(torch, launch, seeds, flush, stream):
    """One launch per seed, L2 flushed before each, each timed alone with
    CUDA events on the launching stream; returns the summed seconds."""
    total = 0.0
    for sd in seeds:
        flush.fill_(sd & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch(sd)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1e3
    return total


def run_rre(args):
    """Batched reaction-rate-equation integration (the deterministic mean-field
    counterpart): the 32 x 64 random network's parameter sweep integrated by
    Dormand-Prince 5(4) with a power-of-two step controller, one warp per
    system, FP64 (bit-exact with the oracle's integration).  Reported:
    integration attempts/s (accepted + rejected steps) and the FP64 roofline
    position; the oracle's rate on a strided sample beside it."""
    import torch

    from paper_1309_7695_b300 import abi

    dev = torch.device("cuda:0")
    b = inputs.random_batch(32, 64, args.rre_sims, seed=0, t_end=args.rre_t_end, n_samples=args.rre_samples,
                            network_seed=0)
    net = b.network
    n, N, S = b.n_sims, net.n_species, len(b.sample_times)
    model = abi.Model(net)
    p = torch.from_numpy(b.params).to(dev)
    x = torch.from_numpy(b.x0).to(dev)
    T = torch.from_numpy(b.sample_times).to(dev)
    out = torch.empty((n, S, N), dtype=torch.float64, device=dev)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def launch(_):
        abi.ssa_integrate_rre_dev(model, p, x, T, out, st, rtol=1e-8, atol=1e-8, max_steps=1_000_000, stream=stream)

    _timed_launches(torch, launch, range(args.warmup), flush, stream)
    clocks = ClockSampler(0)
    clocks.start()
    dt = _timed_launches(torch, launch, range(args.steps), flush, stream)
    clk = clocks.stop()
    s = st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)
    attempts = float(s["attempts"].sum()) * args.steps     # every launch integrates the same systems
    accepted = float(s["leaps"].sum()) * args.steps
    ops = attempts * rre_fp64_ops_per_attempt(net)
    achieved = ops / dt
    peak, rates = measured_fp64_peak()
    line = {"metric": "RRE integration attempts/s (Dormand-Prince 5(4), FP64, bit-exact with the oracle)",
            "workload": "rre", "value": attempts / dt, "unit": "attempts/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "accepted_steps_per_s": accepted / dt, "systems_per_s": n * args.steps / dt,
            "dtype": "f64", "data": "synthetic (seeded random network and parameter sweep)",
            "status_ok": int((s["status"] == 0).sum()), "max_attempts_one_system": int(s["attempts"].max()),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                         "unit": "T FP64-op/s", "frac": achieved / peak, "traffic": None,
                         "ops_per_attempt": rre_fp64_ops_per_attempt(net),
                         "peak_source": "of measured: FP64 add rate of this device (ssa_measure_issue_rates, live)",
                         "nominal_frac": achieved / FP64_NOMINAL_OPS},
            "gpu_launches": args.steps, "clocks": clk,
            "config": {"workload": f"RRE of a random mass-action network 32 species x 64 reactions, {n} parameter "
                                   f"sets (rates logU[1e-4,1], x0 U{{0..1000}}), t_end={args.rre_t_end:g}, {S} sample "
                                   f"times, rtol=atol=1e-8", "l2": "flushed before every launch"}}
    if not args.no_cpu_baseline:
        import oracle

        rows = np.arange(0, n, 16)
        t0 = time.perf_counter()
        _, ost = oracle.rre_simulate(net, b.params[rows], b.x0[rows], b.sample_times, rtol=1e-8, atol=1e-8,
                                     max_steps=1_000_000)
        odt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(ost["attempts"].sum()) / odt, "unit": "attempts/s",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"every 16th system ({len(rows)} of {n})", "seconds": round(odt, 2)}
    model.close()
    print(json.dumps(line), flush=True)
    return 0


def run_cle(args):
    """The Langevin leap against the Poisson leap on a workload where every
    leap mean is large: birth-death 0 -> X (c = 2e5), X -> 0 (c = 1) from
    X = 0 to t_end = 5 (stationary mean 2e5), FP64, one launch per mode,
    same seeds.  Reported: leap attempts/s of each mode and their ratio."""
    import torch

    from paper_1309_7695_b300 import abi

    dev = torch.device("cuda:0")
    b = inputs.replicate_batch(inputs.birth_death(), [2e5, 1.0], [0], args.cle_sims, 5.0, 6)
    n, N, S = b.n_sims, 1, len(b.sample_times)
    model = abi.Model(b.network)
    p = torch.from_numpy(b.params).to(dev)
    x = torch.from_numpy(b.x0).to(dev)
    T = torch.from_numpy(b.sample_times).to(dev)
    out = torch.empty((n, S, N), dtype=torch.int32, device=dev)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for name, mode in (("langevin", abi.SSA_MODE_CLE), ("poisson", abi.SSA_MODE_TAU_LEAP)):
        o = abi.ssa_default_options(mode=mode, layout=abi.SSA_LAYOUT_LANE, max_attempts=1 << 20)

        def launch(sd):
            abi.ssa_simulate_dev(model, p, x, b.t_end, T, out, st, seed=sd, opts=o, stream=stream)

        _timed_launches(torch, launch, [300 + w for w in range(args.warmup)], flush, stream)
        dt, leaps, ssa, fir = 0.0, 0.0, 0.0, 0.0
        for k in range(args.steps):
            dt += _timed_launches(torch, launch, [100 + k], flush, stream)
            s = st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)
            leaps += float(s["leaps"].sum() + s["rejected"].sum())
            ssa += float(s["ssa_steps"].sum())
            fir += float(s["firings"].sum())
        res[name] = {"leap_attempts_per_s": leaps / dt, "sim_steps_per_s": (leaps + ssa) / dt,
                     "firings_per_s": fir / dt, "ms_per_step": dt * 1e3 / args.steps}
    line = {"metric": "leap attempts/s, Langevin vs Poisson leap", "workload": "cle",
            "value": res["langevin"]["leap_attempts_per_s"], "unit": "leap attempts/s",
            "higher_is_better": True, "steps": args.steps, "warmup": args.warmup, "dtype": "f64",
            "data": "synthetic", "langevin": res["langevin"], "poisson": res["poisson"],
            "langevin_vs_poisson": res["langevin"]["leap_attempts_per_s"] / res["poisson"]["leap_attempts_per_s"],
            "gpu_launches": 2 * args.steps,
            "config": {"workload": f"birth-death 0->X (2e5), X->0 (1), X0=0, t_end=5, {S} sample times, "
                                   f"{n} replicates, lane layout", "l2": "flushed before every launch"}}
    model.close()
    print(json.dumps(line), flush=True)
    return 0


# FP64 peak for context: the nominal B300 FP64 rate, 1.25 TFLOP/s, as FP64
# operations with a multiply-add counted once
FP64_NOMINAL_OPS = 1.25e12 / 2


def measured_fp64_peak():
    """The device's FP64 add rate, measured live by the library's issue-rate
    microbenchmark (ssa_measure_issue_rates: a full-device grid of
    independent add chains, best of three launches): the roofline
    denominator of kernels bound by FP64 instruction issue."""
    from paper_1309_7695_b300 import abi

    r = abi.ssa_measure_issue_rates()
    return r["fp64_adds_per_s"], r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--layout", type=int, default=0, help="0 auto, 1 warp per simulation, 2 lane per simulation")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fast"],
                    help="precision of the headline leg (fp64: the reference mode, the reported benchmark)")
    ap.add_argument("--schedule", default="multi", choices=["multi", "streams", "serial"],
                    help="multi: the steps' batches in flight in one persistent launch; streams: one launch per "
                         "batch on its own stream; serial: one launch per batch, one after another")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fast", action="store_true")
    ap.add_argument("--no-moments", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-work-counters", action="store_true",
                    help="skip the untimed replay that counts the method's work (the roofline is then omitted)")
    ap.add_argument("--side-batches", type=int, default=8,
                    help="batches simulated by each side leg (fast, persistent, moments, end to end)")
    ap.add_argument("--served-rate", type=float, default=0.5, help="arrival rate of the short served leg (1/s)")
    ap.add_argument("--served-requests", type=int, default=32)
    # profiling / sweep knobs; the reported benchmark uses the defaults
    ap.add_argument("--sims", type=int, default=None, help="override the simulations per GPU (profiling)")
    ap.add_argument("--cap", type=int, default=None, help="override the per-simulation attempt cap (profiling)")
    ap.add_argument("--workload", default="rand32x64", choices=["rand32x64", "rand128x256", "hetero", "served", "rre", "cle"])
    ap.add_argument("--rre-sims", type=int, default=4096)
    ap.add_argument("--rre-t-end", type=float, default=10.0)
    ap.add_argument("--rre-samples", type=int, default=11)
    ap.add_argument("--cle-sims", type=int, default=16384)
    ap.add_argument("--hetero-sims", type=int, default=20000)
    ap.add_argument("--hetero-no-plain", action="store_true", help="skip the one-launch-per-network comparison")
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--serve-networks", type=int, default=32)
    ap.add_argument("--serve-cap", type=int, default=1 << 18)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10.0, 100.0, 1000.0])
    args = ap.parse_args()
    if args.sims is not None:
        WORKLOAD["n_sims"] = args.sims
    if args.cap is not None:
        WORKLOAD["max_attempts"] = args.cap
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "hetero":
        return run_hetero(args)
    if args.workload == "rand128x256":
        return run_sweep128(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "rre":
        return run_rre(args)
    if args.workload == "cle":
        return run_cle(args)

    import torch
    import torch.distributed as dist

    from paper_1309_7695_b300 import abi, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    def barrier():
        if world > 1:
            dist.barrier()

    batch = make_batch(rank)
    net = batch.network
    N, M, S, n = net.n_species, net.n_reactions, len(batch.sample_times), batch.n_sims
    sim_offset = shard.weak_offset(rank, n)
    model = abi.Model(net)
    p = torch.from_numpy(batch.params).to(dev)
    x = torch.from_numpy(batch.x0).to(dev)
    T = torch.from_numpy(batch.sample_times).to(dev)
    # the side legs (fast mode, persistent, moments, end to end) simulate at
    # most this many batches, so that the whole run stays within minutes
    side_k = min(args.steps, args.side_batches)
    nb = max(args.steps, args.warmup) if args.schedule != "serial" else 1
    nb = max(nb, side_k)
    outs = [torch.empty((n, S, N), dtype=torch.int32, device=dev) for _ in range(nb)]
    sts = [torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev) for _ in range(nb)]
    work = torch.zeros(abi.SSA_WORK_COUNTERS, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    side = [torch.cuda.Stream(device=dev) for _ in range(nb)]

    def options(precision, counted=False):
        return abi.ssa_default_options(eps=WORKLOAD["eps"], n_c=WORKLOAD["n_c"],
                                       max_attempts=WORKLOAD["max_attempts"], layout=args.layout, precision=precision,
                                       work_counters=work.data_ptr() if counted else None)

    def run(seeds, precision, schedule, counted=False):
        """Simulate one batch per seed (the steps); returns (seconds, [stats], launches)."""
        o = options(precision, counted)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats, launches = [], 0
        if schedule == "multi":
            groups = [dict(model=model, params=p, x0=x, sample_times=T, samples=outs[k], stats=sts[k],
                           t_end=batch.t_end, seed=sd, sim_offset=sim_offset) for k, sd in enumerate(seeds)]
            e0.record(stream)
            abi.ssa_simulate_multi_dev(groups, opts=o, stream=stream)
            e1.record(stream)
            launches = 1
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            stats = [sts[k].cpu().numpy().view(abi.STATS_DTYPE).reshape(-1) for k in range(len(seeds))]
        elif schedule == "streams":
            e0.record(stream)
            for k, sd in enumerate(seeds):
                side[k].wait_event(e0)
                abi.ssa_simulate_dev(model, p, x, batch.t_end, T, outs[k], sts[k], seed=sd, opts=o,
                                     sim_offset=sim_offset, stream=side[k])
                stream.wait_stream(side[k])
            e1.record(stream)
            launches = len(seeds)
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            stats = [sts[k].cpu().numpy().view(abi.STATS_DTYPE).reshape(-1) for k in range(len(seeds))]
        else:
            dt = 0.0
            for sd in seeds:
                flush.fill_(sd & 0xFF)
                torch.cuda.synchronize()
                e0.record(stream)
                abi.ssa_simulate_dev(model, p, x, batch.t_end, T, outs[0], sts[0], seed=sd, opts=o,
                                     sim_offset=sim_offset, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                dt += e0.elapsed_time(e1) / 1e3
                stats.append(sts[0].cpu().numpy().view(abi.STATS_DTYPE).reshape(-1).copy())
                launches += 1
        return dt, stats, launches

    def sched_name(schedule):
        return {"multi": f"the {args.steps} steps' batches in flight in one persistent launch",
                "streams": f"one launch per step on {args.steps} concurrent streams",
                "serial": "one launch per step, one after another, L2 flushed between"}[schedule]

    def totals(stats):
        fir = sum(float(s["firings"].sum()) for s in stats)
        steps = sum(float(s["leaps"].sum() + s["ssa_steps"].sum()) for s in stats)
        return fir, steps

    head_prec = abi.SSA_FP64_REF if args.precision == "fp64" else abi.SSA_FAST
    run([5000 + w for w in range(args.warmup)], head_prec, args.schedule)
    peak_ops, issue_rates = measured_fp64_peak()

    # ---- the headline: FP64 reference mode, K batches (work counted in the same launches)
    clocks = ClockSampler(local)
    flush.fill_(1)
    work.zero_()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    local_t, stats, launches = run([1000 + k for k in range(args.steps)], head_prec, args.schedule)
    clk = clocks.stop()
    barrier()
    fir, simsteps = totals(stats)
    # the algorithmic work of the timed batches: the same launches replayed, untimed, with the work
    # counters on (the simulations are deterministic, so the replay does exactly the timed work)
    wk = np.zeros(abi.SSA_WORK_COUNTERS)
    if not args.no_work_counters:
        work.zero_()
        run([1000 + k for k in range(args.steps)], head_prec, args.schedule, counted=True)
        wk = work.cpu().numpy().astype(np.float64)
    ops = sum(algorithmic_fp64_ops(s, wk / len(stats), net) for s in stats)
    capped = sum(int((s["status"] == abi.SSA_STATUS_STEP_LIMIT).sum()) for s in stats)
    t_max, (fir, simsteps, ops, capped) = shard.reduce_run(local_t, [fir, simsteps, ops, capped], device=dev)

    # ---- the target comparison: the plain one-launch-per-batch FP64 kernel against the
    # fast form in one persistent launch (the fast form's accuracy against FP64: the coupled
    # KS / moment tests)
    plain = None
    if not args.no_fast:
        # two batches, one launch each: a single batch's time is its tail of long simulations,
        # which varies from run to run with the warps they happen to share
        per = []
        for sd in (3000, 3001):
            pt, pstats, _ = run([sd], abi.SSA_FP64_REF, "serial")
            pf, ps = totals(pstats)
            pt, (pf, ps) = shard.reduce_run(pt, [pf, ps], device=dev)
            per.append((pt, pf, ps))
        pt = sum(v[0] for v in per)
        pf = sum(v[1] for v in per)
        ps = sum(v[2] for v in per)
        plain = {"value": pf / pt, "unit": "firings/s", "sim_steps_per_s": ps / pt,
                 "seconds_per_batch": [round(v[0], 3) for v in per],
                 "schedule": "one batch per launch, launches one after another, L2 flushed before each (2 batches)"}
    fast = None
    fast_persistent = None
    if not args.no_fast:
        # fast mode on the headline's batches and schedule, for the precision comparison
        ft, fstats, _ = run([1000 + k for k in range(args.steps)], abi.SSA_FAST, args.schedule)
        ff, fsteps = totals(fstats)
        ft, (ff, fsteps) = shard.reduce_run(ft, [ff, fsteps], device=dev)
        fast = {"value": ff / ft, "unit": "firings/s", "sim_steps_per_s": fsteps / ft,
                "ms_per_step": ft * 1e3 / args.steps, "batches": args.steps, "schedule": sched_name(args.schedule),
                "vs_fp64": (ff / ft) / (fir / t_max), "dtype": "f32 propensities/Poisson, f64 clock/a0/tau'"}
        seeds = [1000 + k for k in range(side_k)]
        mt, mstats, _ = run(seeds, abi.SSA_FAST, "multi")
        mf, msteps = totals(mstats)
        work.zero_()
        run(seeds, abi.SSA_FAST, "multi", counted=True)
        mwk = work.cpu().numpy().astype(np.float64)
        mops = sum(algorithmic_fp64_ops(s, mwk / len(mstats), net) for s in mstats)
        mt, (mf, msteps, mops) = shard.reduce_run(mt, [mf, msteps, mops], device=dev)
        fast_persistent = {"value": mf / mt, "unit": "firings/s", "sim_steps_per_s": msteps / mt,
                           "ms_per_step": mt * 1e3 / side_k, "batches": side_k,
                           "schedule": f"the {side_k} batches in one persistent launch",
                           "vs_plain_fp64": (mf / mt) / plain["value"] if plain else None,
                           "roofline": {"bound": "alu", "achieved": mops / mt / 1e12, "peak": peak_ops / 1e12,
                                        "unit": "T FP64-op/s (method ops at FP64 rate)",
                                        "frac": mops / mt / peak_ops, "peak_source": "of measured (live)",
                                        "traffic": TRAFFIC_BYTES_PER_SIM["FastArith"] * side_k * n,
                                        "traffic_source": TRAFFIC_SOURCE},
                           "dtype": "f32 propensities/Poisson, f64 clock/a0/tau'"}

    moments = None
    if not args.no_moments:
        # the same batches with sweep moments accumulated on the device instead of
        # trajectories written (ssa_simulate_moments_dev), batches in flight on streams
        o = options(abi.SSA_FP64_REF)
        means = [torch.empty((S, N), dtype=torch.float64, device=dev) for _ in range(side_k)]
        varis = [torch.empty((S, N), dtype=torch.float64, device=dev) for _ in range(side_k)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(side_k):
            side[k].wait_event(e0)
            abi.ssa_simulate_moments_dev(model, p, x, batch.t_end, T, means[k], varis[k], sts[k], seed=1000 + k,
                                         opts=o, sim_offset=sim_offset, stream=side[k])
            stream.wait_stream(side[k])
        e1.record(stream)
        torch.cuda.synchronize()
        mt = e0.elapsed_time(e1) / 1e3
        mf = sum(float(sts[k].cpu().numpy().view(abi.STATS_DTYPE)["firings"].sum()) for k in range(side_k))
        mt, (mf,) = shard.reduce_run(mt, [mf], device=dev)
        moments = {"value": mf / mt, "unit": "firings/s", "ms_per_step": mt * 1e3 / side_k, "batches": side_k,
                   "schedule": f"one launch per batch on its own stream ({side_k} streams), not the headline's "
                               "persistent launch",
                   "output_bytes_per_step": int(2 * S * N * 8), "trajectory_bytes_per_step": int(n * S * N * 4)}

    e2e = None
    if not args.no_e2e:
        # host-buffer path: pinned inputs -> ssa_submit_batch (H2D inside, one job and stream per
        # step, all in flight together) -> ssa_fetch (D2H) of every step's samples and counters
        hp = torch.from_numpy(batch.params).pin_memory().numpy()
        hx = torch.from_numpy(batch.x0).pin_memory().numpy()
        hT = batch.sample_times.copy()
        hs = [torch.empty((n, S, N), dtype=torch.int32).pin_memory().numpy() for _ in range(side_k)]
        hst = [np.zeros(n, dtype=abi.STATS_DTYPE) for _ in range(side_k)]
        o = options(abi.SSA_FP64_REF)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        jobs = [abi.ssa_submit_batch(model, hp, hx, batch.t_end, hT, seed=1000 + k, opts=o) for k in range(side_k)]
        for k, job in enumerate(jobs):
            job.fetch(hs[k], hst[k])
        e2e_t = time.perf_counter() - t0
        for job in jobs:
            job.release()
        e2e_f = sum(float(h["firings"].sum()) for h in hst)
        e2e_t, (e2e_f,) = shard.reduce_run(e2e_t, [e2e_f], device=dev)
        e2e = {"value": e2e_f / e2e_t, "unit": "firings/s", "batches": side_k,
               "h2d_bytes_per_step": int(hp.nbytes + hx.nbytes + hT.nbytes),
               "d2h_bytes_per_step": int(hs[0].nbytes + hst[0].nbytes),
               "schedule": "one ssa_submit_batch job (own stream) per step, all in flight"}

    served = None
    if not args.no_served and world == 1:
        res = served_stream([args.served_rate], args.served_requests, args.serve_networks, args.serve_cap)[0]
        served = {**res, "config": served_config(args.served_requests, args.serve_networks, args.serve_cap),
                  "note": "arrival rate chosen below the measured service capacity of this stream"}

    if rank == 0:
        kernel_s = local_t / launches
        achieved = ops / world / launches / kernel_s
        sched = sched_name(args.schedule)
        line = {"metric": METRIC, "value": fir / t_max, "unit": "firings/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32 propensities/Poisson, f64 clock/a0/tau'",
                "data": "synthetic (seeded random network and parameter sweep)",
                "sim_steps_per_s": simsteps / t_max,
                "config": config_dict({"parallelism": f"dp{world} (independent simulation shards)",
                                       "precision": "fp64-ref" if args.precision == "fp64" else "fast",
                                       "capped_fraction": capped / (world * n * args.steps), "schedule": sched,
                                       "l2": "each step reads 41 MB of inputs and writes 847 MB of samples (> L2); "
                                             "L2 flushed before the timed region"}),
                "roofline": None if args.no_work_counters else {
                             "bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                             "unit": "T FP64-op/s", "frac": achieved / peak_ops,
                             "traffic": traffic_per_launch(args, args.precision, n), "traffic_source": TRAFFIC_SOURCE,
                             "kernel": kernel_name(args),
                             "peak_source": "of measured: FP64 add rate of this device, measured live by "
                                            "ssa_measure_issue_rates",
                             "nominal_frac": achieved / FP64_NOMINAL_OPS,
                             "fp32_adds_per_s": issue_rates["fp32_adds_per_s"],
                             "fp64_add_latency_cycles": issue_rates["fp64_add_latency_cycles"],
                             "ops_per_batch": ops / (world * args.steps),
                             "work_counters_per_batch": {nm: float(v) / args.steps for nm, v in zip(abi.WORK_NAMES, wk)}},
                "clocks": clk, "gpu_launches": launches, "e2e": e2e, "plain_fp64": plain, "fast_mode": fast,
                "fast_persistent": fast_persistent, "served": served, "moments_mode": moments}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_rate(batch, gpu_stats=stats[0])
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    model.close()
    return 0

if __name__ == "__main__":
    sys.exit(main())
