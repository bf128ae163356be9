"""Measured launch shapes for the fine kernel.

`tune(problems)` groups the problems by precision and by power-of-two
bucket of P, measures each bucket once with `mmp_autotune` (one saturated
fine launch per candidate quads-per-thread count, the bucket's largest
problem, a few steps per slice), and registers the fastest count for the
bucket with `mmp_set_tuning`; single-problem contexts created afterwards
use it when their slices fill the GPU.  `tune_batch(problems)` measures the
cap on quads per thread of a batch (one batched sweep of a sample per
candidate) and registers it with `mmp_set_batch_nq`.  Results are cached in
a JSON file keyed by GPU name and library version (`cache`, else
$MMP_TUNE_CACHE, else no file); a cached entry is registered without
measuring.
"""
from __future__ import annotations

import json
import math
import os

from . import mmp
from . import workloads as W


def _bucket(P: int) -> int:
    return int(math.floor(math.log2(max(1, P))))


def _device_key() -> str:
    import torch

    return f"{torch.cuda.get_device_name(0)}|libmmp {mmp.load().mmp_version()}"


def tune(problems: list[W.Problem] | W.Problem, cache: str | None = None, probe_steps: int = 0,
         candidates=None) -> dict:
    """Measure (or load) and register the quads per thread of every
    (precision, P bucket) among `problems`; returns {"prec:bucket": {...}}."""
    if isinstance(problems, W.Problem):
        problems = [problems]
    path = cache if cache is not None else os.environ.get("MMP_TUNE_CACHE")
    store = {}
    if path and os.path.exists(path):
        with open(path) as f:
            store = json.load(f)
    dev = _device_key()
    table = store.setdefault(dev, {})
    groups: dict[str, W.Problem] = {}
    for p in problems:
        key = f"{p.precision}:{_bucket(p.P)}"
        rep = groups.get(key)
        if rep is None or (p.P, p.N) > (rep.P, rep.N):
            groups[key] = p
    out = {}
    for key, rep in sorted(groups.items()):
        prec, b = key.split(":")
        b = int(b)
        entry = table.get(key)
        if entry is None:
            r = mmp.mmp_autotune(rep, candidates=candidates, probe_steps=probe_steps)
            entry = {"nq": r["best_nq"], "rates": {str(k): v for k, v in r["rates"].items()},
                     "probe": {"P": rep.P, "N": rep.N}}
            table[key] = entry
        mmp.mmp_set_tuning(prec, 2 ** b, 2 ** (b + 1) - 1, entry["nq"])
        out[key] = entry
    if path:
        with open(path, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
    return out


def tune_batch(problems: list[W.Problem], candidates=(13, 17, 20, 23, 26, 27), sample: int = 64,
               cache: str | None = None) -> dict:
    """Measure the batch cap on quads per thread: for each candidate, one
    batched sweep (all slices) of an evenly strided sample of `problems`,
    timed with CUDA events; the fastest cap is registered with
    mmp_set_batch_nq for batched contexts created afterwards.  Returns
    {"nq": best, "rates": {cap: particle-steps/s}, "sample": n}."""
    import torch

    prec = problems[0].precision
    path = cache if cache is not None else os.environ.get("MMP_TUNE_CACHE")
    store = {}
    if path and os.path.exists(path):
        with open(path) as f:
            store = json.load(f)
    table = store.setdefault(_device_key(), {})
    key = f"batch:{prec}:{len(problems)}"
    entry = table.get(key)
    if entry is None:
        stride = max(1, len(problems) // sample)
        sub = problems[::stride][:sample]
        rates = {}
        for cap in [candidates[0]] + list(candidates):  # the first run warms the kernels up
            mmp.mmp_set_batch_nq(prec, cap)
            s = mmp.Solver(sub)
            mmp.mmp_set_timing(s.ctx, True)
            s.lift()
            torch.cuda.synchronize()
            mmp.mmp_timing(s.ctx, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.iterate(1)
            e1.record()
            torch.cuda.synchronize()
            steps = mmp.mmp_timing(s.ctx, reset=True)["fine_particle_steps"]
            rates[str(cap)] = steps / (e0.elapsed_time(e1) / 1e3)
            s.close()
        best = max(candidates, key=lambda c: rates[str(c)])
        entry = {"nq": best, "rates": rates, "sample": len(sub)}
        table[key] = entry
        if path:
            with open(path, "w") as f:
                json.dump(store, f, indent=1, sort_keys=True)
    mmp.mmp_set_batch_nq(prec, entry["nq"])
    return entry


def clear() -> None:
    """Remove every registered entry and batch cap (both precisions)."""
    for prec in ("mixed", "fp64"):
        mmp.mmp_set_tuning(prec, 0, 0, 0)
        mmp.mmp_set_batch_nq(prec, 0)
