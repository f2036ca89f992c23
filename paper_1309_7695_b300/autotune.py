"""Launch-shape autotuner and multi-network scheduler.

The kernels take four shape choices that change speed but never results:
the layout (one simulation per lane for SSA steps with warp-cooperative
leaps, or one warp per simulation), the warps per CTA (which sets shared
memory per CTA and so occupancy), how many lanes of a warp own a
simulation (fewer spread heavy simulations over more warps, so their
warp-cooperative leaps do not queue behind each other), and the register
budget of the kernel build (up to 255 registers per thread, or 168 so that
a third 4-warp CTA fits on an SM when shared memory allows).  ``tune`` times
short trial launches of the candidates on a strided sample of the batch
(attempt cap lowered so a trial takes milliseconds) and keeps the fastest
by attempts per second; results are cached per device and network shape.

``plan`` orders the groups of a multi-network launch by their measured
per-simulation cost, most expensive first, so the long simulations start
early and overlap the rest instead of forming the tail, and picks the
launch shape for the mixed workload.

All measurements go through the C ABI; nothing here computes a simulation.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import abi

CACHE_ENV = "TAULEAP_TUNE_CACHE"
# (warps per CTA, simulations per warp, register budget: 0 = up to 255, 1 = 168)
LANE_CANDIDATES = [(2, 32, 0), (4, 32, 0), (8, 32, 0), (4, 16, 0), (4, 8, 0), (8, 4, 0), (4, 32, 1), (2, 32, 1),
                   (4, 16, 1)]


def _cache_path() -> str:
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache", "tauleap", "tune.json")


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _key(network, precision, mode, device_name):
    nnz = int((network.stoichiometry() != 0).sum())
    return f"{device_name}|N{network.n_species}|M{network.n_reactions}|nnz{nnz}|p{precision}|m{mode}"


def _sample_rows(n, k):
    stride = max(1, n // k)
    return np.arange(0, n, stride)[:k]


def _trial(model, p, x, T, t_end, opts, seed, torch):
    n = int(p.shape[0])
    out = torch.empty((n, int(T.numel()), model.n_species), dtype=torch.int32, device=p.device)
    st = torch.empty((n, abi.STATS_DTYPE.itemsize), dtype=torch.uint8, device=p.device)
    abi.ssa_simulate_dev(model, p, x, t_end, T, out, st, seed=seed, opts=opts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    abi.ssa_simulate_dev(model, p, x, t_end, T, out, st, seed=seed, opts=opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s = st.cpu().numpy().view(abi.STATS_DTYPE).reshape(-1)
    return float(s["attempts"].sum()) / max(dt, 1e-9), dt


def tune(network, model, params, x0, sample_times, t_end, precision=abi.SSA_FP64_REF,
         mode=abi.SSA_MODE_TAU_LEAP, sample=2048, trial_cap=4096, seed=12345, use_cache=True):
    """Pick (layout, block_warps, sims_per_warp, reg_cap) for one network.

    params/x0/sample_times: torch CUDA tensors of the batch (a strided
    sample of ``sample`` rows is timed).  Returns a dict with the chosen
    option values and the measured attempts/s of every candidate."""
    import torch

    dev_name = torch.cuda.get_device_name(params.device)
    key = _key(network, precision, mode, dev_name)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    rows = torch.from_numpy(_sample_rows(int(params.shape[0]), sample)).to(params.device)
    p, x = params.index_select(0, rows).contiguous(), x0.index_select(0, rows).contiguous()
    results = []
    cands = [(abi.SSA_LAYOUT_LANE, bw, spw, rc) for bw, spw, rc in LANE_CANDIDATES]
    if precision == abi.SSA_FP64_REF:
        cands.append((abi.SSA_LAYOUT_WARP, 4, 0, 0))
    for layout, bw, spw, rc in cands:
        o = abi.ssa_default_options(precision=precision, mode=mode, max_attempts=trial_cap, layout=layout,
                                    block_warps=bw, sims_per_warp=spw, reg_cap=rc)
        try:
            rate, dt = _trial(model, p, x, sample_times, t_end, o, seed, torch)
        except abi.SsaError:
            continue
        results.append({"layout": layout, "block_warps": bw, "sims_per_warp": spw, "reg_cap": rc,
                        "attempts_per_s": rate})
    best = max(results, key=lambda r: r["attempts_per_s"])
    entry = {"layout": best["layout"], "block_warps": best["block_warps"], "sims_per_warp": best["sims_per_warp"],
             "reg_cap": best["reg_cap"], "candidates": results}
    if use_cache:
        cache[key] = entry
        _store_cache(cache)
    return entry


def apply(opts, entry):
    """Copy a tuning result into an ssa_options structure."""
    opts.layout = entry["layout"]
    opts.block_warps = entry["block_warps"]
    opts.sims_per_warp = entry["sims_per_warp"]
    opts.reg_cap = entry.get("reg_cap", 0)
    return opts


def plan(groups, precision=abi.SSA_FAST, mode=abi.SSA_MODE_TAU_LEAP, sample=64, trial_cap=4096, seed=54321):
    """Schedule for one multi-network launch.

    groups: list of dicts as taken by abi.ssa_simulate_multi_dev.  Each
    group's per-simulation cost is measured on ``sample`` strided rows with
    the attempt cap lowered to ``trial_cap``; the groups are returned most
    expensive first, with launch options tuned on a trial of the mixed
    workload.  Returns (ordered_groups, options, costs)."""
    import torch

    costs = []
    for g in groups:
        n = int(g["params"].shape[0])
        rows = torch.from_numpy(_sample_rows(n, sample)).to(g["params"].device)
        p = g["params"].index_select(0, rows).contiguous()
        x = g["x0"].index_select(0, rows).contiguous()
        o = abi.ssa_default_options(precision=precision, mode=mode, max_attempts=trial_cap)
        _, dt = _trial(g["model"], p, x, g["sample_times"], g["t_end"], o, seed, torch)
        costs.append(dt / max(1, int(rows.numel())))
    order = sorted(range(len(groups)), key=lambda k: -costs[k])
    ordered = [groups[k] for k in order]
    # launch shape for the mixed workload: trial on a strided subset of every group
    best, best_rate = None, -1.0
    for bw, spw, rc in LANE_CANDIDATES:
        trial = []
        for g in ordered:
            n = int(g["params"].shape[0])
            rows = torch.from_numpy(_sample_rows(n, max(8, sample // 4))).to(g["params"].device)
            m = int(rows.numel())
            trial.append(dict(g, params=g["params"].index_select(0, rows).contiguous(),
                              x0=g["x0"].index_select(0, rows).contiguous(),
                              samples=torch.empty((m, int(g["sample_times"].numel()), g["model"].n_species),
                                                  dtype=torch.int32, device=g["params"].device),
                              stats=torch.empty((m, abi.STATS_DTYPE.itemsize), dtype=torch.uint8,
                                                device=g["params"].device)))
        o = abi.ssa_default_options(precision=precision, mode=mode, max_attempts=trial_cap, block_warps=bw,
                                    sims_per_warp=spw, reg_cap=rc)
        try:
            abi.ssa_simulate_multi_dev(trial, opts=o)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            abi.ssa_simulate_multi_dev(trial, opts=o)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        except abi.SsaError:
            continue
        att = sum(float(t["stats"].cpu().numpy().view(abi.STATS_DTYPE)["attempts"].sum()) for t in trial)
        rate = att / max(dt, 1e-9)
        if rate > best_rate:
            best, best_rate = (bw, spw, rc), rate
    opts = abi.ssa_default_options(precision=precision, mode=mode, block_warps=best[0], sims_per_warp=best[1],
                                   reg_cap=best[2])
    return ordered, opts, [costs[k] for k in order]
