"""The parallel CPU baseline (OpenMP) of the PaRSorting++ refine step, for
timing against the GPU on the host's cores.  Benchmark infrastructure only:
the library never imports it.  build() compiles par_sorting.c with gcc."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "libpar_sorting.so")
_lib = None


def build() -> str:
    src = os.path.join(HERE, "par_sorting.c")
    if os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(src):
        return SO
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    tmp = SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, SO)
    return SO


def _l():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p, i64 = ctypes.c_void_p, ctypes.c_int64
        _lib.par_sorting_run.argtypes = [i64, p, p, i64, ctypes.c_int, p, p]
    return _lib


def run(g, T: int, threads: int = 0):
    """PaRSorting++ T iterations from zero loads: (loads, (edges, vertices, iteration))."""
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32) if g.adj.size else np.zeros(1, np.int32)
    loads = np.zeros(g.n, np.int64)
    best = np.zeros(3, np.int64)
    if _l().par_sorting_run(g.n, off.ctypes.data, adj.ctypes.data, T, threads, loads.ctypes.data,
                            best.ctypes.data) != 0:
        raise MemoryError("par_sorting_run")
    return loads, tuple(int(x) for x in best)


def threads() -> int:
    return os.cpu_count() or 1
