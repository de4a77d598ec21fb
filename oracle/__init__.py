"""CPU oracle for the load-weighted peeling of Greedy++ (arXiv 2311.04333).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are the only callers.  The product path
(the CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``oracle.c`` (plain sequential C, exact integers);
this module compiles it with gcc and exposes it through ctypes:

  * ``run(g, variant, T, p, q, init_loads)`` -- T iterations of Alg. 2 with the
    ordering of GreedySorting++ (variant 0, Sec. 3.2), ParallelGreedy++ round
    peeling with eps = p/q (variant 1, Sec. 3.3) or sequential Greedy++
    (variant 2); returns final loads, best (edges, vertices), best iteration,
    best vertex set and the per-iteration trace;
  * ``iteration(...)`` -- one iteration with its order and deg* exposed;
  * ``sorting_order``, ``round_order``, ``load_order`` -- the orderings O;
  * ``brute_force``, ``maxflow_densest``, ``coreness``,
    ``coreness_by_deletion`` -- exact checkers used to pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib_handle = None

SORTING, PEELING, GREEDY = 0, 1, 2


def build() -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "oracle.c")
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        # DSG_ORACLE_SO lets the mutation test load a deliberately broken copy
        lib = ctypes.CDLL(os.environ.get("DSG_ORACLE_SO") or build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_sorting_order.argtypes = [i64, p, p]
        lib.oracle_round_order.argtypes = [i64, p, p, p, i64, i64, p, p, p]
        lib.oracle_round_order.restype = i64
        lib.oracle_load_order.argtypes = [i64, p, p, p, p]
        lib.oracle_peel_iteration.argtypes = [i64, p, p, p, p, p, p, p, p, p, p]
        lib.oracle_run.argtypes = [i64, p, p, ctypes.c_int, i64, i64, i64, p, p, p, p, p]
        lib.oracle_brute_force.argtypes = [i64, p, p, p]
        lib.oracle_maxflow_densest.argtypes = [i64, p, p, p, p]
        lib.oracle_coreness.argtypes = [i64, p, p, p]
        lib.oracle_coreness_by_deletion.argtypes = [i64, p, p, p]
        lib.oracle_run_pruned.argtypes = [i64, p, p, ctypes.c_int, i64, i64, i64, p, p, p, p, p]
        lib.oracle_run_pruned_c.argtypes = [i64, p, p, ctypes.c_int, i64, i64, i64, i64, i64, p, p, p, p, p]
        lib.oracle_run_pruned_ax.argtypes = [i64, p, p, ctypes.c_int, i64, i64, i64, i64, i64, p, p, p, p, p]
        lib.oracle_apx_coreness.argtypes = [i64, p, p, i64, i64, p]
        lib.oracle_core_subgraph.argtypes = [i64, p, p, p, i64, p, p]
        _lib_handle = lib
    return _lib_handle


def _p(a) -> int | None:
    return None if a is None else a.ctypes.data


def _csr(g):
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    return int(g.n), off, adj


@dataclass
class Result:
    loads: np.ndarray        # int64[n]
    best_edges: int
    best_vertices: int
    best_iter: int           # 0: S = G never beaten
    best_pos: int            # position of the best suffix in its iteration
    best_set: np.ndarray     # int64 ascending ids
    trace: np.ndarray        # int64[T, 3]: iteration's densest suffix (e, v), width


def run(g, variant: int = SORTING, T: int = 1, p: int = 0, q: int = 1,
        init_loads=None) -> Result:
    n, off, adj = _csr(g)
    loads = np.zeros(n, dtype=np.int64)
    best = np.zeros(5, dtype=np.int64)
    bset = np.zeros(n, dtype=np.int64)
    trace = np.zeros((max(T, 1), 3), dtype=np.int64)
    il = None if init_loads is None else np.ascontiguousarray(init_loads, dtype=np.int64)
    rc = _lib().oracle_run(n, _p(off), _p(adj), variant, T, p, q, _p(il), _p(loads),
                           _p(best), _p(bset), _p(trace))
    if rc != 0:
        raise ValueError(f"oracle_run failed with status {rc}")
    return Result(loads, int(best[0]), int(best[1]), int(best[2]), int(best[4]),
                  bset[: best[3]].copy(), trace[:T].copy())


def sorting_order(loads) -> np.ndarray:
    loads = np.ascontiguousarray(loads, dtype=np.int64)
    order = np.zeros(loads.shape[0], dtype=np.int64)
    _lib().oracle_sorting_order(loads.shape[0], _p(loads), _p(order))
    return order


def round_order(g, loads, p: int, q: int):
    """ParallelGreedy++ order: (order, round_of, round_min[:rounds])."""
    n, off, adj = _csr(g)
    loads = np.ascontiguousarray(loads, dtype=np.int64)
    order = np.zeros(n, dtype=np.int64)
    rnd = np.zeros(n, dtype=np.int64)
    rmin = np.zeros(n + 1, dtype=np.int64)
    r = _lib().oracle_round_order(n, _p(off), _p(adj), _p(loads), p, q, _p(order), _p(rnd), _p(rmin))
    if r < 0:
        raise ValueError("oracle_round_order failed")
    return order, rnd, rmin[:r].copy()


def load_order(g, loads) -> np.ndarray:
    n, off, adj = _csr(g)
    loads = np.ascontiguousarray(loads, dtype=np.int64)
    order = np.zeros(n, dtype=np.int64)
    _lib().oracle_load_order(n, _p(off), _p(adj), _p(loads), _p(order))
    return order


def iteration(g, order, loads, best=None):
    """One Alg. 2 iteration over a given order.  Returns a dict with the new
    loads, deg* by position, the iteration's densest suffix (e, v, pos), the
    running best and the position where it improved (-1 if it did not)."""
    n, off, adj = _csr(g)
    order = np.ascontiguousarray(order, dtype=np.int64)
    loads = np.array(loads, dtype=np.int64, copy=True)
    degstar = np.zeros(n, dtype=np.int64)
    it_best = np.zeros(3, dtype=np.int64)
    be = ctypes.c_int64(best[0] if best else int(off[-1]) // 2)
    bv = ctypes.c_int64(best[1] if best else n)
    at = ctypes.c_int64(-1)
    w = ctypes.c_int64(0)
    _lib().oracle_peel_iteration(n, _p(off), _p(adj), _p(order), _p(loads), _p(degstar),
                                 _p(it_best), ctypes.addressof(be), ctypes.addressof(bv),
                                 ctypes.addressof(at), ctypes.addressof(w))
    return dict(loads=loads, degstar=degstar, it_best=tuple(int(x) for x in it_best),
                best=(be.value, bv.value), improved_at=at.value, width=w.value)


def brute_force(g):
    """Densest subgraph by enumeration (n <= 24): (edges, vertices, mask)."""
    n, off, adj = _csr(g)
    out = np.zeros(3, dtype=np.int64)
    if _lib().oracle_brute_force(n, _p(off), _p(adj), _p(out)) != 0:
        raise ValueError("brute force needs 1 <= n <= 24")
    return int(out[0]), int(out[1]), int(out[2])


def maxflow_densest(g):
    """Exact densest subgraph by parametric min cut: ((edges, vertices), mask)."""
    n, off, adj = _csr(g)
    out = np.zeros(2, dtype=np.int64)
    side = np.zeros(n, dtype=np.uint8)
    if _lib().oracle_maxflow_densest(n, _p(off), _p(adj), _p(out), _p(side)) != 0:
        raise ValueError("maxflow failed")
    return (int(out[0]), int(out[1])), side.astype(bool)


def coreness(g) -> np.ndarray:
    n, off, adj = _csr(g)
    core = np.zeros(n, dtype=np.int64)
    _lib().oracle_coreness(n, _p(off), _p(adj), _p(core))
    return core


def coreness_by_deletion(g) -> np.ndarray:
    n, off, adj = _csr(g)
    core = np.zeros(n, dtype=np.int64)
    _lib().oracle_coreness_by_deletion(n, _p(off), _p(adj), _p(core))
    return core


@dataclass
class PrunedResult:
    loads: np.ndarray
    best_edges: int
    best_vertices: int
    best_iter: int
    best_set: np.ndarray
    trace: np.ndarray        # [T, 3]: refine result (edges, vertices), vertices of the G it ran on
    k_max: int
    core_vertices: int       # |V| of the ceil(k_max/2)-core
    core_edges: int
    final_vertices: int      # |V| of the final G
    L: tuple                 # final lower bound (numerator, denominator)


def apx_coreness(g, c: tuple = (3, 2)) -> np.ndarray:
    """c-approximate core numbers (c = c[0] / c[1] > 1): the smallest level
    tau_i >= core(v) of tau_0 = 1, tau_{i+1} = ceil(tau_i * c); 0 for core 0."""
    n, off, adj = _csr(g)
    out = np.zeros(n, dtype=np.int64)
    if _lib().oracle_apx_coreness(n, _p(off), _p(adj), c[0], c[1], _p(out)) != 0:
        raise ValueError("oracle_apx_coreness failed")
    return out


def run_pruned(g, variant: int = SORTING, T: int = 1, p: int = 0, q: int = 1, c: tuple = None) -> PrunedResult:
    """Alg. 1 (Pruning-and-Refining) with `variant` as Refine: exact pruning,
    or with c = (c_num, c_den) pruning by the c-approximate decomposition
    (k_max of the result is then k-hat_max)."""
    n, off, adj = _csr(g)
    loads = np.zeros(n, dtype=np.int64)
    best = np.zeros(5, dtype=np.int64)
    bset = np.zeros(n, dtype=np.int64)
    trace = np.zeros((max(T, 1), 3), dtype=np.int64)
    info = np.zeros(6, dtype=np.int64)
    cn, cd = c if c else (0, 1)
    rc = _lib().oracle_run_pruned_c(n, _p(off), _p(adj), variant, T, p, q, cn, cd, _p(loads), _p(best),
                                    _p(bset), _p(trace), _p(info))
    if rc != 0:
        raise ValueError(f"oracle_run_pruned_c failed with status {rc}")
    return PrunedResult(loads, int(best[0]), int(best[1]), int(best[2]), bset[: best[3]].copy(), trace[:T].copy(),
                        int(info[0]), int(info[1]), int(info[2]), int(info[3]), (int(info[4]), int(info[5])))


def run_pruned_apx_exact(g, variant: int = PEELING, T: int = 1, p: int = 0, q: int = 1,
                         c: tuple = (3, 2)) -> tuple:
    """PaRApxGreedy++'s pruning (Sec. 4): approximate pruning by the
    c-approximate decomposition to G1 = {k-hat >= ceil(k-hat_max / (2c))},
    then Alg. 1 with exact pruning on G1.  Returns (PrunedResult, k-hat_max,
    |V(G1)|, |E(G1)|); k_max and the core sizes in the result are G1's."""
    n, off, adj = _csr(g)
    loads = np.zeros(n, dtype=np.int64)
    best = np.zeros(5, dtype=np.int64)
    bset = np.zeros(n, dtype=np.int64)
    trace = np.zeros((max(T, 1), 3), dtype=np.int64)
    info = np.zeros(9, dtype=np.int64)
    rc = _lib().oracle_run_pruned_ax(n, _p(off), _p(adj), variant, T, p, q, c[0], c[1], _p(loads), _p(best),
                                     _p(bset), _p(trace), _p(info))
    if rc != 0:
        raise ValueError(f"oracle_run_pruned_ax failed with status {rc}")
    r = PrunedResult(loads, int(best[0]), int(best[1]), int(best[2]), bset[: best[3]].copy(), trace[:T].copy(),
                     int(info[0]), int(info[1]), int(info[2]), int(info[3]), (int(info[4]), int(info[5])))
    return r, int(info[6]), int(info[7]), int(info[8])


def core_subgraph_size(g, core, k: int) -> tuple:
    """(|V|, |E|) of the subgraph induced on {v : core[v] >= k}."""
    n, off, adj = _csr(g)
    core = np.ascontiguousarray(core, dtype=np.int64)
    nn = np.zeros(1, dtype=np.int64)
    mm = np.zeros(1, dtype=np.int64)
    if _lib().oracle_core_subgraph(n, _p(off), _p(adj), _p(core), k, _p(nn), _p(mm)) != 0:
        raise ValueError("oracle_core_subgraph failed")
    return int(nn[0]), int(mm[0])
