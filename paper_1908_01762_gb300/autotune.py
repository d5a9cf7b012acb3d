"""Autotuner of the launch shapes: tile size (threads per block), Verlet skin
and the PPE sweeps' synchronisation form.

None of the three changes what a step computes beyond rounding: the skin only
changes how often the cell sort and skin lists are rebuilt (the refreshed
neighbour sets are the same), the tile size regroups the per-tile FP32 sums of
the convergence test, and the two sweep forms give the same bits.  They do
change the time: larger tiles mean fewer, longer per-tile chains; a wider skin
means fewer rebuilds but longer lists to filter at every refresh; the
point-to-point sweeps save the grid barriers only while every block owns one
tile.

`tune` times graph-replayed steps of the caller's own workload (L2 flushed
between steps, CUDA events on the library's stream; as many steps as the run
to be tuned, since the PPE's sweep count changes as a flow develops) for every
candidate and keeps the fastest, unless it beats the defaults by less than 1 %.  Results are cached in a JSON file per GPU
model and workload class (dimension, precision, case count and total size to
within a factor of about 1.4, walls or not); `lookup` returns the cached
options for a workload of the same class.  The package ships the cache tuned
on GB300 for the benchmark workloads.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import sisph

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_gb300.json")
BLOCKS = (128, 256)
SKINS = (0.10, 0.15, 0.25)
DEFAULTS = {"block": 256, "skin": 0.15, "ppe_sync": 0}
L2_FLUSH_BYTES = 256 << 20


def workload_key(cases, precision, device):
    """Cache key: the GPU model and the workload class."""
    n = int(sum(int(c["n"]) for c in cases))
    nc = len(cases)
    walls = any(bool(np.any(np.asarray(c["kind"]) != 0)) for c in cases)
    cls = 1 if nc == 1 else 2 ** math.ceil(math.log2(nc))
    size = int(round(2.0 * math.log2(max(n, 1))))        # half-octaves of the total size
    prec = "mixed" if precision == sisph.MIXED else "fp64"
    return f"{device}|dim{int(cases[0]['dim'])}|{prec}|cases{cls}|n2^{size / 2:g}|walls{int(walls)}"


def candidates(cases, sms):
    """The option sets to time.  The barrier form is tried against the
    automatic choice only where the automatic choice can be the point-to-point
    form (at most a few fluid tiles per SM); elsewhere both are the barrier."""
    out = []
    for block in BLOCKS:
        tiles = sum(-(-int(np.sum(np.asarray(c["kind"]) == 0)) // block) for c in cases)
        syncs = (0,) if tiles > 8 * sms else (0, 1)
        for skin in SKINS:
            for sync in syncs:
                out.append({"block": block, "skin": skin, "ppe_sync": sync})
    return out


def load_cache(path):
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def store(path, key, entry):
    """Merge one entry into the cache file (written whole, then renamed)."""
    data = load_cache(path)
    data[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def device_name():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name} sm_{p.major}{p.minor} x{p.multi_processor_count}"


def lookup(cases, precision, path=DEFAULT_CACHE, device=None):
    """Cached options for this workload class on this GPU, or None."""
    key = workload_key(cases, precision, device or device_name())
    entry = load_cache(path).get(key)
    return None if entry is None else dict(entry["options"])


def time_options(cases, precision, opts, steps, warmup, flush, stream):
    """Mean device time per step (ms) of `steps` replayed steps after `warmup`
    ones, or None if the handle cannot be made or a step fails."""
    import torch
    try:
        sim = sisph.Simulation(cases, precision=precision, use_graph=1, **opts)
    except sisph.SisphError:
        return None
    try:
        sisph.sisph_set_stream(sim.h, stream.cuda_stream)
        for _ in range(warmup):
            sim.step(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in ev)) / steps
    except sisph.SisphError:
        return None
    finally:
        sim.close()


def pick(trials, margin=0.01):
    """The fastest trial that ran (ties keep the earlier one), unless it is
    less than `margin` faster than the first trial (the defaults): a gain
    within run-to-run noise does not move the choice off the defaults."""
    ok = [t for t in trials if t["ms_per_step"] is not None]
    if not ok:
        raise RuntimeError("no candidate ran")
    best = min(ok, key=lambda t: t["ms_per_step"])
    first = trials[0]
    if first["ms_per_step"] is not None and best["ms_per_step"] > first["ms_per_step"] * (1.0 - margin):
        return first
    return best


def tune(cases, precision, steps=30, warmup=3, path=None, log=None, timer=None, device=None,
         sms=None):
    """Time every candidate (the defaults first) on `cases` and return the
    cache entry {options, ms_per_step, default_ms_per_step, trials}, merged
    into the cache file at `path` when given.  `timer(options)` -> ms per step
    or None replaces the GPU timing (with `device` and `sms` given too)."""
    if timer is None:
        import torch
        dev = torch.device("cuda")
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        device = device_name()

        def timer(opts):
            return time_options(cases, precision, opts, steps, warmup, flush, stream)
    cands = [dict(DEFAULTS)] + [c for c in candidates(cases, sms) if c != DEFAULTS]
    trials = []
    for opts in cands:
        ms = timer(opts)
        trials.append({"options": opts, "ms_per_step": ms})
        if log:
            log(f"autotune {opts}: {ms if ms is None else round(ms, 4)} ms/step")
    best = pick(trials)
    entry = {"options": best["options"], "ms_per_step": best["ms_per_step"],
             "default_ms_per_step": trials[0]["ms_per_step"], "steps": steps, "trials": trials}
    if path:
        store(path, workload_key(cases, precision, device), entry)
    return entry
