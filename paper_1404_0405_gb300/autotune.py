"""Self-written autotuner for the ensemble step: patch side and work-list grid.

Times a short ensemble run (CUDA events, after warm-up) for every pair of patch
side p (the element layout and the work-list granularity) and blocks per SM of
the work-list launches, on the caller's workload, and returns the fastest pair in
active-cell steps per second.  Results are cached per (GPU, workload key) in
``_build/tune.json`` next to the library.  Argument marshalling and loop control
only: every step runs in the library's kernels.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import Model, step_ensemble
from .buildlib import OUT_DIR

CACHE = os.path.join(OUT_DIR, "tune.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def _live(m):
    return sum(m.stats()["live_nodes"].values())


def tune(jmin, jmax, eps, fields_of, members=4, precision="fp32", patches=(4, 8, 16), blocks=(2, 4, 8), steps=3,
         warmup=2, key_extra="", use_cache=True, persistent=False):
    """fields_of(xyz, edges) -> list of (dh, u) initial states (one per member) on a
    grid with the given node and edge order; persistent: the members' stage mode
    (see Model).  Returns ({"patch", "blocks_per_sm", "rate"}, table of every
    trial)."""
    import torch
    key = f"{_gpu_name()}|J{jmin}-{jmax}|eps{eps:g}|M{members}|{precision}|{persistent}|{key_extra}"
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]["best"], cache[key]["trials"]
    trials = []
    for p in patches:
        base = Model(jmin, jmax, patch=p, eps=eps)
        xyz, en = base.grid(jmax)
        states = fields_of(xyz, en)[:members]
        for b in blocks:
            ms = []
            for dh, u in states:
                m = Model(jmin, jmax, patch=p, eps=eps, share=base, blocks_per_sm=b, precision=precision,
                          persistent=persistent)
                m.set_state(dh, u)
                m.adapt()
                ms.append(m)
            step_ensemble(ms, -1.0, warmup, True)
            torch.cuda.synchronize()
            cells0 = sum(_live(m) for m in ms)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step_ensemble(ms, -1.0, steps, True)
            e1.record()
            torch.cuda.synchronize()
            cells = 0.5 * (cells0 + sum(_live(m) for m in ms)) * steps
            rate = cells / (e0.elapsed_time(e1) / 1e3)
            trials.append({"patch": p, "blocks_per_sm": b, "rate": rate})
            for m in ms:
                m.close()
        base.close()
    best = max(trials, key=lambda t: t["rate"])
    cache[key] = {"best": best, "trials": trials}
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return best, trials
