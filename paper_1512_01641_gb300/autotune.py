"""Autotuner of the planner's fill knobs (tile width, tiling threshold).

The batched fill cuts large pairs into 32-row x ``tile_cols`` tiles (pairs of
at least ``tile_min_cells`` cells) and runs small pairs whole, one warp each.
The best knobs depend on the GPU and on the batch's size distribution (how
many long pairs, how long), so they are measured: every candidate is applied
to the plan (mine_plan_set_option), the fill is timed with CUDA events on the
launching stream, and the fastest is kept.  Results are cached in a JSON file
keyed by the GPU name and a histogram of the pairs' sizes (log2 of N and M).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

from . import miner

CANDIDATES = {"tile_cols": [32, 64, 128], "tile_min_cells": [1 << 16, 1 << 17, 1 << 18, 1 << 20]}
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gb300_miner", "autotune.json")


def shape_key(batch) -> str:
    """GPU name + a histogram of (ceil log2 N, ceil log2 M) over the pairs."""
    import torch
    N = np.maximum(batch.src.doc_sizes(), 1)
    M = np.maximum(batch.tgt.doc_sizes(), 1)
    h = np.zeros((16, 16), np.int64)
    np.add.at(h, (np.minimum(np.ceil(np.log2(N)).astype(int), 15), np.minimum(np.ceil(np.log2(M)).astype(int), 15)), 1)
    # coarse: fractions of pairs per bin, rounded, so that reseeded batches of
    # the same shape share an entry
    frac = np.round(h / max(batch.n_pairs, 1), 3)
    digest = hashlib.sha1(frac.tobytes() + str(batch.n_pairs // 1000).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name()}|{digest}"


def _time_fill(plan, params, counts, reps):
    plan.set_timing(True)
    for _ in range(reps):
        plan.align(params, counts)
    kt = plan.kernel_times()
    plan.set_timing(False)
    return kt["fill"][0] / max(kt["fill"][1], 1)


def autotune(plan: "miner.Plan", batch, params: "miner.MineParams", counts=None, reps: int = 2,
             cache_path: str | None = CACHE, candidates=CANDIDATES) -> dict:
    """Pick the fastest fill knobs for this plan, apply them, return a report."""
    key = shape_key(batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        best = cache[key]["best"]
        for k, v in best.items():
            plan.set_option(k, v)
        return {"cached": True, "key": key, **cache[key]}
    if counts is None:
        counts = plan.count()
    trials = []
    names = list(candidates)
    for combo in itertools.product(*(candidates[n] for n in names)):
        knobs = dict(zip(names, combo))
        for k, v in knobs.items():
            plan.set_option(k, v)
        _time_fill(plan, params, counts, 1)  # warm
        trials.append((_time_fill(plan, params, counts, reps), knobs))
    trials.sort(key=lambda x: x[0])
    best = trials[0][1]
    for k, v in best.items():
        plan.set_option(k, v)
    rec = {"best": best, "fill_ms": trials[0][0], "trials": [{"fill_ms": t, **k} for t, k in trials]}
    if cache_path:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache[key] = rec
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"cached": False, "key": key, **rec}
