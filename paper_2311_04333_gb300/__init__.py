"""GB300-native densest subgraph refinement: PaRSorting++ and PaRGreedy++
(arXiv 2311.04333), per-iteration load-weighted peeling of Greedy++.

The compute path is libdsg (hand-written sm_103a CUDA behind the C ABI of
include/dsg.h); this package is its Python binding.  Importing it loads the
library and raises if it is missing or was not built: there is no CPU path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._dsg import (DSG_ERR_BUSY, DSG_ERR_CUDA, DSG_ERR_INVALID, DSG_ERR_NOMEM, DSG_ERR_OVERFLOW,
                   DSG_ERR_TIMEOUT, DSG_OK, DSG_DST_DEVICE, DSG_INIT_DEVICE, DSG_PATH_BLOCK, DSG_PATH_GRID, DSG_NOALLOC_MAX_VERTICES, DSG_PEELING,
                   DSG_SORTING, DSG_SRC_DEVICE, DSG_VALIDATE, DsgError, LIB_PATH, dsg_create,
                   dsg_batch_info, dsg_densest_suffix_noalloc, dsg_destroy, dsg_free_batch, dsg_set_batch_tuning,
                   dsg_free_graph, dsg_run_batch, dsg_coreness, dsg_apx_coreness, dsg_run_pruned, dsg_run_pruned_apx, dsg_run_pruned_apx_exact, dsg_server_create, dsg_server_destroy,
                   dsg_server_stats, dsg_server_submit, dsg_server_wait, dsg_upload_batch,
                   dsg_get_stats, dsg_get_peel_stats, dsg_graph_info, dsg_last_error, dsg_run, dsg_set_profiling,
                   dsg_upload_csr, dsg_debug_set, DSG_DEBUG_SPIN_LIMIT, DSG_DEBUG_STALL,
                   DSG_DEBUG_FAIL_ALLOC, DSG_DEBUG_FAIL_UPLOAD, DSG_DEBUG_PEEL_BLOCKS)

__all__ = ["DSG_OK", "DSG_ERR_INVALID", "DSG_ERR_NOMEM", "DSG_ERR_CUDA", "DSG_ERR_OVERFLOW",
           "DSG_ERR_TIMEOUT", "DSG_ERR_BUSY", "DSG_PATH_GRID", "DSG_PATH_BLOCK", "DSG_SORTING", "DSG_PEELING", "DSG_VALIDATE", "DSG_SRC_DEVICE", "DSG_DST_DEVICE",
           "DSG_INIT_DEVICE", "DsgError", "LIB_PATH", "dsg_create", "dsg_destroy",
           "dsg_free_graph", "dsg_get_stats", "dsg_get_peel_stats", "dsg_graph_info", "dsg_last_error", "dsg_run",
           "dsg_set_profiling", "dsg_upload_csr", "dsg_densest_suffix_noalloc",
           "DSG_NOALLOC_MAX_VERTICES", "dsg_upload_batch", "dsg_batch_info", "dsg_run_batch",
           "dsg_free_batch", "dsg_set_batch_tuning", "dsg_coreness", "dsg_apx_coreness", "dsg_run_pruned", "dsg_run_pruned_apx", "dsg_run_pruned_apx_exact", "dsg_server_create", "dsg_server_submit", "dsg_server_wait",
           "dsg_server_stats", "dsg_server_destroy", "Result", "densest", "dsg_debug_set",
           "DSG_DEBUG_SPIN_LIMIT", "DSG_DEBUG_STALL", "DSG_DEBUG_FAIL_ALLOC", "DSG_DEBUG_FAIL_UPLOAD",
           "DSG_DEBUG_PEEL_BLOCKS"]


@dataclass
class Result:
    best_edges: int
    best_vertices: int
    best_iter: int
    best_set: np.ndarray      # int32 ascending ids
    loads: np.ndarray         # int64[n]
    trace: np.ndarray         # int64[T, 3]


def densest(ctx, n: int, offsets: np.ndarray, adj: np.ndarray, variant: int = DSG_SORTING,
            T: int = 10, eps: tuple[int, int] = (1, 10), init_loads=None,
            validate: bool = True, path: int = 0) -> Result:
    """Upload a host CSR graph, run T refine iterations and read back."""
    g = dsg_upload_csr(ctx, n, offsets, adj, DSG_VALIDATE if validate else 0)
    try:
        loads = np.zeros(n, dtype=np.int64)
        bset = np.zeros(n, dtype=np.int32)
        trace = np.zeros(3 * T, dtype=np.int64)
        r = dsg_run(ctx, g, variant, T, eps[0], eps[1], init_loads, loads, bset, trace, path)
    finally:
        dsg_free_graph(g)
    return Result(r["best_edges"], r["best_vertices"], r["best_iter"],
                  bset[: r["best_set_size"]].copy(), loads, trace.reshape(T, 3))
