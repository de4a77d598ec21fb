"""Autotuner for the batched launch.  It picks, by timing each candidate on the
batch itself, the knobs of dsg_run_batch / dsg_set_batch_tuning:

  * threads per graph (the block size one graph gets): 256, 512 or 1024;
  * PaRSorting++: the list length below which a vertex's arcs are scanned by
    one thread instead of a warp (thread_degree);
  * PaRGreedy++: the degree above which a round's peeled vertex is counted by
    the whole block instead of a warp (block_degree).

The search is coordinate-wise: block size first with the default degree,
then the degree knob at the chosen block size.  The choice is cached per GPU
name, batch shape class (number of graphs and total edges, rounded to powers
of two) and variant in a JSON file.  The run it times is the same
dsg_run_batch call the caller makes; results do not depend on the knobs."""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import _dsg

CANDIDATES = (256, 512, 1024)
THREAD_DEGREES = (8, 16, 32, 64, 128)
BLOCK_DEGREES = (256, 1024, 4096)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def _shape_class(G: int, total_m: int) -> str:
    return f"G2^{max(0, math.ceil(math.log2(max(G, 1))))}_m2^{max(0, math.ceil(math.log2(max(total_m, 1))))}"


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def apply(ctx, batch, rec: dict) -> int:
    """Set a tuning record's degree knobs on the batch; returns its block size."""
    _dsg.dsg_set_batch_tuning(ctx, batch, int(rec.get("thread_degree", 0)), int(rec.get("block_degree", 0)))
    return int(rec["threads"])


def tune_batch(ctx, batch, T, cache_path: str | None = DEFAULT_CACHE, reps: int = 1,
               candidates=CANDIDATES, force: bool = False, variant: int = _dsg.DSG_SORTING,
               eps_num=None, eps_den=None, degrees=None) -> dict:
    """Returns {"threads", "thread_degree", "block_degree", "ms": {candidate:
    ms}} and records it; the batch is left tuned to the choice."""
    G, N, M = _dsg.dsg_batch_info(batch)
    key = f"{_gpu_name()}|{_shape_class(G, M)}|variant{variant}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache and "threads" in cache[key]:
        apply(ctx, batch, cache[key])
        return cache[key]
    knob = "block_degree" if variant == _dsg.DSG_PEELING else "thread_degree"
    if degrees is None:
        degrees = BLOCK_DEGREES if variant == _dsg.DSG_PEELING else THREAD_DEGREES
    best = np.zeros(4 * G, np.int64)
    times = {}

    def timed(th: int, deg: int) -> float:
        _dsg.dsg_set_batch_tuning(ctx, batch, deg if knob == "thread_degree" else 0,
                                  deg if knob == "block_degree" else 0)
        _dsg.dsg_run_batch(ctx, batch, variant, T, th, best, eps_num=eps_num, eps_den=eps_den)   # warm
        t0 = time.perf_counter()
        for _ in range(reps):
            _dsg.dsg_run_batch(ctx, batch, variant, T, th, best, eps_num=eps_num, eps_den=eps_den)
        ms = (time.perf_counter() - t0) / reps * 1e3
        times[f"{th}/{deg}"] = ms
        return ms

    default_deg = 1024 if knob == "block_degree" else 32
    by_threads = {th: timed(th, default_deg) for th in candidates}
    th_best = min(by_threads, key=by_threads.get)
    by_deg = {default_deg: by_threads[th_best]}
    for d in degrees:
        if d != default_deg:
            by_deg[d] = timed(th_best, d)
    d_best = min(by_deg, key=by_deg.get)
    rec = {"threads": th_best, knob: d_best, "ms": times, "shape": _shape_class(G, M)}
    apply(ctx, batch, rec)
    cache[key] = rec
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return rec
