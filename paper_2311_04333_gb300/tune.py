"""Autotuner for the batched launch: picks the thread-block size that one
graph of the batch gets (256, 512 or 1024 threads) by timing each candidate
on the batch itself, and caches the choice per GPU name and batch shape class
(number of graphs and total edges, rounded to powers of two) in a JSON file.
The run it times is the same dsg_run_batch call the caller makes."""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import _dsg

CANDIDATES = (256, 512, 1024)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def _shape_class(G: int, total_m: int) -> str:
    return f"G2^{max(0, math.ceil(math.log2(max(G, 1))))}_m2^{max(0, math.ceil(math.log2(max(total_m, 1))))}"


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def tune_batch(ctx, batch, T, cache_path: str | None = DEFAULT_CACHE, reps: int = 1,
               candidates=CANDIDATES, force: bool = False, variant: int = _dsg.DSG_SORTING,
               eps_num=None, eps_den=None) -> dict:
    """Returns {"threads": best, "ms": {candidate: time}} and records it."""
    G, N, M = _dsg.dsg_batch_info(batch)
    key = f"{_gpu_name()}|{_shape_class(G, M)}|variant{variant}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        return cache[key]
    best = np.zeros(4 * G, np.int64)
    times = {}
    for th in candidates:
        _dsg.dsg_run_batch(ctx, batch, variant, T, th, best, eps_num=eps_num, eps_den=eps_den)  # warm
        t0 = time.perf_counter()
        for _ in range(reps):
            _dsg.dsg_run_batch(ctx, batch, variant, T, th, best, eps_num=eps_num, eps_den=eps_den)
        times[th] = (time.perf_counter() - t0) / reps * 1e3
    rec = {"threads": min(times, key=times.get), "ms": times, "shape": _shape_class(G, M)}
    cache[key] = rec
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return rec
