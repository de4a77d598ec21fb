"""ctypes binding of libdsg (include/dsg.h): argument marshalling only.

Every function keeps the C name.  Arrays may be numpy arrays (host memory)
or torch tensors (host or CUDA); the binding passes their data pointers and
sets DSG_SRC_DEVICE / DSG_DST_DEVICE / DSG_INIT_DEVICE from where they live.
All computation happens in libdsg's CUDA kernels; if the library cannot be
loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DSG_OK, DSG_ERR_INVALID, DSG_ERR_NOMEM, DSG_ERR_CUDA, DSG_ERR_OVERFLOW, DSG_ERR_TIMEOUT, DSG_ERR_BUSY = range(7)
DSG_SORTING, DSG_PEELING = 0, 1
DSG_VALIDATE, DSG_SRC_DEVICE = 0x1, 0x2
DSG_DST_DEVICE, DSG_INIT_DEVICE = 0x1, 0x2
DSG_PATH_GRID, DSG_PATH_BLOCK = 0x4, 0x8
DSG_PHASE_EDGE_SCAN, DSG_PHASE_SORT, DSG_PHASE_OTHER, DSG_PHASE_COUNT = 0, 1, 2, 3

STATUS_NAMES = {0: "DSG_OK", 1: "DSG_ERR_INVALID", 2: "DSG_ERR_NOMEM", 3: "DSG_ERR_CUDA",
                4: "DSG_ERR_OVERFLOW", 5: "DSG_ERR_TIMEOUT", 6: "DSG_ERR_BUSY"}


class DsgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class dsg_result(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("best_iter", ctypes.c_int32),
                ("best_edges", ctypes.c_int64), ("best_vertices", ctypes.c_int64),
                ("best_set_size", ctypes.c_int64), ("loads", ctypes.c_void_p),
                ("best_set", ctypes.c_void_p), ("trace", ctypes.c_void_p)]


class dsg_prune_info(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int64), ("core_vertices", ctypes.c_int64), ("core_edges", ctypes.c_int64),
                ("final_vertices", ctypes.c_int64), ("L_num", ctypes.c_int64), ("L_den", ctypes.c_int64)]


class dsg_server_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("best_iter", ctypes.c_int32),
                ("best_edges", ctypes.c_int64), ("best_vertices", ctypes.c_int64),
                ("best_set_size", ctypes.c_int64), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("slot", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("error", ctypes.c_char * 256)]


class dsg_batch_result(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("best", ctypes.c_void_p), ("loads", ctypes.c_void_p),
                ("sets", ctypes.c_void_p), ("trace", ctypes.c_void_p)]


def _load():
    path = os.environ.get("DSG_LIB") or _build.build()
    lib = ctypes.CDLL(path)
    P, I64, I32, U32, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int
    lib.dsg_create.argtypes = [I, P, ctypes.POINTER(P)]
    lib.dsg_destroy.argtypes = [P]
    lib.dsg_destroy.restype = None
    lib.dsg_last_error.argtypes = [P]
    lib.dsg_last_error.restype = ctypes.c_char_p
    lib.dsg_debug_set.argtypes = [P, I, I64]
    lib.dsg_upload_csr.argtypes = [P, I64, P, P, U32, ctypes.POINTER(P)]
    lib.dsg_graph_info.argtypes = [P, P, P, P]
    lib.dsg_run.argtypes = [P, I, I32, I64, I64, P, ctypes.POINTER(dsg_result)]
    lib.dsg_free_graph.argtypes = [P]
    lib.dsg_free_graph.restype = None
    lib.dsg_set_profiling.argtypes = [P, I]
    lib.dsg_get_stats.argtypes = [P, P, P, P, I]
    lib.dsg_get_peel_stats.argtypes = [P, P, P, P, I]
    lib.dsg_densest_suffix_noalloc.argtypes = [P, P, I64, I64, P, P]
    lib.dsg_upload_batch.argtypes = [P, I32, P, P, P, U32, ctypes.POINTER(P)]
    lib.dsg_batch_info.argtypes = [P, P, P, P]
    lib.dsg_run_batch.argtypes = [P, I, P, P, P, I32, ctypes.POINTER(dsg_batch_result)]
    lib.dsg_set_batch_tuning.argtypes = [P, I32, I32]
    lib.dsg_free_batch.argtypes = [P]
    lib.dsg_free_batch.restype = None
    lib.dsg_coreness.argtypes = [P, P, ctypes.POINTER(I64), ctypes.c_uint32]
    lib.dsg_run_pruned.argtypes = [P, I, I32, I64, I64, ctypes.POINTER(dsg_result), ctypes.POINTER(dsg_prune_info)]
    lib.dsg_run_pruned_apx.argtypes = [P, I, I32, I64, I64, I64, I64, ctypes.POINTER(dsg_result),
                                       ctypes.POINTER(dsg_prune_info)]
    lib.dsg_run_pruned_apx_exact.argtypes = [P, I, I32, I64, I64, I64, I64, ctypes.POINTER(dsg_result),
                                             ctypes.POINTER(dsg_prune_info)]
    lib.dsg_apx_coreness.argtypes = [P, I64, I64, P, ctypes.POINTER(I64), ctypes.c_uint32]
    lib.dsg_server_create.argtypes = [I, I32, I64, ctypes.POINTER(P)]
    lib.dsg_server_submit.argtypes = [P, I64, P, P, I, I32, I64, I64, ctypes.POINTER(ctypes.c_uint64)]
    lib.dsg_server_wait.argtypes = [P, ctypes.c_uint64, I64, ctypes.POINTER(dsg_server_result), P, P]
    lib.dsg_server_stats.argtypes = [P, P, P, P, P, P]
    lib.dsg_server_destroy.argtypes = [P]
    lib.dsg_server_destroy.restype = None
    return lib


LIB = _load()
LIB_PATH = LIB._name


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype) -> tuple[int | None, bool]:
    """(data pointer, is_device) of a numpy array or torch tensor of `dtype`."""
    if x is None:
        return None, False
    if _is_torch(x):
        import torch
        tdt = {np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return x.data_ptr(), x.is_cuda
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"expected a contiguous numpy {np.dtype(dtype)} array")
    return x.ctypes.data, False


def _count(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(x.size)


def _need(x, count: int, what: str) -> None:
    """The C call reads or writes `count` entries of x: refuse a smaller
    buffer here rather than let the library run past its end."""
    if x is not None and _count(x) < count:
        raise ValueError(f"{what} holds {_count(x)} entries; the call uses {count}")


def _graph_n(graph) -> int | None:
    """Vertex count of an uploaded graph (None for a handle the library
    rejects; the call itself then reports that)."""
    n = ctypes.c_int64()
    return n.value if LIB.dsg_graph_info(graph, ctypes.byref(n), None, None) == DSG_OK else None


def _check(ctx, rc: int) -> None:
    if rc != DSG_OK:
        raise DsgError(rc, LIB.dsg_last_error(ctx).decode())


def dsg_create(device: int = 0, stream: int | None = None):
    """Create a context on `device`; `stream` is a cudaStream_t handle (int)."""
    out = ctypes.c_void_p()
    rc = LIB.dsg_create(device, stream, ctypes.byref(out))
    if rc != DSG_OK:
        raise DsgError(rc, f"dsg_create(device={device}) failed")
    return out.value


def dsg_destroy(ctx) -> None:
    LIB.dsg_destroy(ctx)


def dsg_last_error(ctx) -> str:
    return LIB.dsg_last_error(ctx).decode()


DSG_DEBUG_SPIN_LIMIT, DSG_DEBUG_STALL, DSG_DEBUG_FAIL_ALLOC, DSG_DEBUG_FAIL_UPLOAD = 1, 2, 3, 4
DSG_DEBUG_PEEL_BLOCKS = 5


def dsg_debug_set(ctx, knob: int, value: int) -> None:
    """Test-only fault hooks (see dsg.h): spin limit and stalled waits per
    context, allocation / upload failure countdowns process-wide."""
    rc = LIB.dsg_debug_set(ctx, knob, value)
    if rc != DSG_OK:
        raise DsgError(rc, f"dsg_debug_set(knob={knob}, value={value})")


def dsg_upload_csr(ctx, n: int, offsets, adj, flags: int = 0):
    po, do = _ptr(offsets, np.int64)
    pa, da = _ptr(adj, np.int32)
    _need(offsets, max(int(n), 0) + 1, "offsets")
    if not do and n >= 0:
        _need(adj, int(offsets[n]), "adj")
    if do != da and pa is not None and int(offsets[-1]) > 0:
        raise ValueError("offsets and adj must both live on the host or both on the device")
    if do:
        flags |= DSG_SRC_DEVICE
    out = ctypes.c_void_p()
    _check(ctx, LIB.dsg_upload_csr(ctx, n, po, pa, flags, ctypes.byref(out)))
    return out.value


def dsg_graph_info(graph) -> tuple[int, int, int]:
    n, m, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = LIB.dsg_graph_info(graph, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d))
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_graph_info")
    return n.value, m.value, d.value


def _need_run_buffers(graph, T, loads, best_set, trace, init_loads=None) -> None:
    n = _graph_n(graph)
    if n is not None:
        _need(loads, n, "loads")
        _need(best_set, n, "best_set")
        _need(init_loads, n, "init_loads")
    _need(trace, 3 * max(int(T), 0), "trace")


def dsg_run(ctx, graph, variant: int, T: int, eps_num: int = 0, eps_den: int = 1,
            init_loads=None, loads=None, best_set=None, trace=None, path: int = 0) -> dict:
    """Run T iterations.  `loads` (int64[n]), `best_set` (int32[n]) and
    `trace` (int64[T*3]) are optional output buffers, all on the host or all
    on the device; `init_loads` (int64[n]) may live on either side.  `path`:
    0 (by size), DSG_PATH_GRID or DSG_PATH_BLOCK."""
    res = dsg_result()
    pl, dl = _ptr(loads, np.int64)
    ps, ds = _ptr(best_set, np.int32)
    pt, dt = _ptr(trace, np.int64)
    pi, di = _ptr(init_loads, np.int64)
    _need_run_buffers(graph, T, loads, best_set, trace, init_loads)
    dev = {d for p, d in ((pl, dl), (ps, ds), (pt, dt)) if p is not None}
    if len(dev) > 1:
        raise ValueError("output buffers must all be host or all device")
    res.flags = (DSG_DST_DEVICE if dev == {True} else 0) | (DSG_INIT_DEVICE if di else 0) | path
    res.loads, res.best_set, res.trace = pl, ps, pt
    _check(ctx, LIB.dsg_run(graph, variant, T, eps_num, eps_den, pi, ctypes.byref(res)))
    return dict(best_edges=res.best_edges, best_vertices=res.best_vertices,
                best_iter=res.best_iter, best_set_size=res.best_set_size)


def dsg_coreness(ctx, graph, core=None) -> tuple:
    """Core numbers (int32[n], host or device buffer; allocated on the host
    when None) and k_max."""
    if core is None:
        n = ctypes.c_int64()
        LIB.dsg_graph_info(graph, ctypes.byref(n), None, None)
        core = np.zeros(n.value, dtype=np.int32)
    pc, dc = _ptr(core, np.int32)
    n = _graph_n(graph)
    if n is not None:
        _need(core, n, "core")
    km = ctypes.c_int64()
    _check(ctx, LIB.dsg_coreness(graph, pc, ctypes.byref(km), DSG_DST_DEVICE if dc else 0))
    return core, km.value


def dsg_apx_coreness(ctx, graph, c=(3, 2), core=None) -> tuple:
    """c-approximate core numbers (int32[n], host or device buffer; allocated
    on the host when None) and their maximum; c = (c_num, c_den)."""
    if core is None:
        n = ctypes.c_int64()
        LIB.dsg_graph_info(graph, ctypes.byref(n), None, None)
        core = np.zeros(n.value, dtype=np.int32)
    pc, dc = _ptr(core, np.int32)
    n = _graph_n(graph)
    if n is not None:
        _need(core, n, "core")
    km = ctypes.c_int64()
    _check(ctx, LIB.dsg_apx_coreness(graph, c[0], c[1], pc, ctypes.byref(km), DSG_DST_DEVICE if dc else 0))
    return core, km.value


def dsg_run_pruned(ctx, graph, variant: int, T: int, eps_num: int = 0, eps_den: int = 1, loads=None,
                   best_set=None, trace=None, c=None, exact_after: bool = False) -> dict:
    """Alg. 1 with `variant` as the refine step; outputs as dsg_run plus the
    pruning info.  c = (c_num, c_den) prunes by the c-approximate core
    numbers (dsg_run_pruned_apx) instead of the exact ones; with exact_after
    the approximate pruning is followed by exact pruning
    (dsg_run_pruned_apx_exact)."""
    res = dsg_result()
    pl, dl = _ptr(loads, np.int64)
    ps, ds = _ptr(best_set, np.int32)
    pt, dt = _ptr(trace, np.int64)
    _need_run_buffers(graph, T, loads, best_set, trace)
    dev = {d for p, d in ((pl, dl), (ps, ds), (pt, dt)) if p is not None}
    if len(dev) > 1:
        raise ValueError("output buffers must all be host or all device")
    res.flags = DSG_DST_DEVICE if dev == {True} else 0
    res.loads, res.best_set, res.trace = pl, ps, pt
    info = dsg_prune_info()
    if c is None:
        _check(ctx, LIB.dsg_run_pruned(graph, variant, T, eps_num, eps_den, ctypes.byref(res), ctypes.byref(info)))
    elif exact_after:
        _check(ctx, LIB.dsg_run_pruned_apx_exact(graph, variant, T, eps_num, eps_den, c[0], c[1], ctypes.byref(res),
                                                 ctypes.byref(info)))
    else:
        _check(ctx, LIB.dsg_run_pruned_apx(graph, variant, T, eps_num, eps_den, c[0], c[1], ctypes.byref(res),
                                           ctypes.byref(info)))
    out = dict(best_edges=res.best_edges, best_vertices=res.best_vertices, best_iter=res.best_iter,
               best_set_size=res.best_set_size)
    out.update({f: getattr(info, f) for f, _ in dsg_prune_info._fields_})
    return out


def dsg_run_pruned_apx(ctx, graph, variant: int, T: int, eps_num: int = 0, eps_den: int = 1, c_num: int = 3,
                       c_den: int = 2, loads=None, best_set=None, trace=None) -> dict:
    """Alg. 1 with pruning by the c-approximate core numbers, c = c_num / c_den."""
    return dsg_run_pruned(ctx, graph, variant, T, eps_num, eps_den, loads, best_set, trace, c=(c_num, c_den))


def dsg_run_pruned_apx_exact(ctx, graph, variant: int, T: int, eps_num: int = 0, eps_den: int = 1, c_num: int = 3,
                             c_den: int = 2, loads=None, best_set=None, trace=None) -> dict:
    """Alg. 1 with approximate pruning followed by exact pruning
    (PaRApxGreedy++ with DSG_PEELING), c = c_num / c_den."""
    return dsg_run_pruned(ctx, graph, variant, T, eps_num, eps_den, loads, best_set, trace, c=(c_num, c_den),
                          exact_after=True)


def dsg_free_graph(graph) -> None:
    LIB.dsg_free_graph(graph)


def dsg_set_profiling(ctx, on: bool) -> None:
    _check(ctx, LIB.dsg_set_profiling(ctx, int(bool(on))))


def dsg_get_stats(ctx, reset: bool = False) -> dict:
    ms = (ctypes.c_double * DSG_PHASE_COUNT)()
    la = (ctypes.c_int64 * DSG_PHASE_COUNT)()
    by = (ctypes.c_int64 * DSG_PHASE_COUNT)()
    _check(ctx, LIB.dsg_get_stats(ctx, ms, la, by, int(bool(reset))))
    names = ["edge_scan", "sort", "other"]
    return {nm: dict(ms=ms[i], launches=la[i], bytes=by[i]) for i, nm in enumerate(names)}


def dsg_get_peel_stats(ctx, reset: bool = False) -> dict:
    """Whole-GPU PaRGreedy++ telemetry: iterations, rounds, alive vertices
    summed over the rounds."""
    it, rd, wk = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, LIB.dsg_get_peel_stats(ctx, ctypes.byref(it), ctypes.byref(rd), ctypes.byref(wk), int(reset)))
    return {"iterations": it.value, "rounds": rd.value, "alive_sum": wk.value}


def dsg_densest_suffix_noalloc(loads, A, n: int, m: int, result, stream: int | None = None) -> None:
    """Enqueue the allocation-free densest-suffix computation.  loads/A are
    uint32 (or int32 bit patterns) CUDA tensors of n entries; result is an
    int64 CUDA tensor of 5 entries; nothing is synchronised."""
    for t in (loads, A, result):
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise TypeError("dsg_densest_suffix_noalloc takes contiguous CUDA tensors")
    rc = LIB.dsg_densest_suffix_noalloc(loads.data_ptr(), A.data_ptr(), n, m, result.data_ptr(), stream)
    if rc != DSG_OK:
        raise DsgError(rc, f"dsg_densest_suffix_noalloc(n={n}, m={m}) failed "
                           f"(n must be in [1, {DSG_NOALLOC_MAX_VERTICES}], m in [0, 2^48))")


def dsg_upload_batch(ctx, graphs, flags: int = 0):
    """graphs: sequence of (n, offsets int64[n+1], adj int32[2m]) host arrays."""
    G = len(graphs)
    n_per = np.array([int(g[0]) for g in graphs], dtype=np.int64)
    offs = [np.ascontiguousarray(g[1], dtype=np.int64) for g in graphs]
    adjs = [np.ascontiguousarray(g[2], dtype=np.int32) for g in graphs]
    poff = (ctypes.c_void_p * G)(*[o.ctypes.data for o in offs])
    padj = (ctypes.c_void_p * G)(*[a.ctypes.data for a in adjs])
    out = ctypes.c_void_p()
    _check(ctx, LIB.dsg_upload_batch(ctx, G, n_per.ctypes.data, poff, padj, flags, ctypes.byref(out)))
    return out.value


def dsg_batch_info(batch) -> tuple[int, int, int]:
    G, n, m = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    rc = LIB.dsg_batch_info(batch, ctypes.byref(G), ctypes.byref(n), ctypes.byref(m))
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_batch_info")
    return G.value, n.value, m.value


def dsg_run_batch(ctx, batch, variant: int, T, threads_per_graph: int = 0, best=None, loads=None,
                  sets=None, trace=None, eps_num=None, eps_den=None) -> None:
    """T: int32[G]; best: int64[4G] (required); loads int64[N], sets int32[N],
    trace int64[3*G*Tmax] optional; all host or all device.  eps_num/eps_den:
    int64[G] (or scalars) for DSG_PEELING, default 0/1."""
    T = np.ascontiguousarray(T, dtype=np.int32)
    G = T.size
    en = None if eps_num is None else np.ascontiguousarray(np.broadcast_to(eps_num, (G,)), dtype=np.int64)
    ed = None if eps_den is None else np.ascontiguousarray(np.broadcast_to(eps_den, (G,)), dtype=np.int64)
    res = dsg_batch_result()
    pb, db = _ptr(best, np.int64)
    pl, dl = _ptr(loads, np.int64)
    ps, ds = _ptr(sets, np.int32)
    pt, dt = _ptr(trace, np.int64)
    Gb, N = ctypes.c_int32(), ctypes.c_int64()
    if LIB.dsg_batch_info(batch, ctypes.byref(Gb), ctypes.byref(N), None) == DSG_OK:
        G = Gb.value
        _need(T, G, "T")
        _need(best, 4 * G, "best")
        _need(loads, N.value, "loads")
        _need(sets, N.value, "sets")
        _need(trace, 3 * G * max(int(T[:G].max()), 0), "trace")
    dev = {d for p, d in ((pb, db), (pl, dl), (ps, ds), (pt, dt)) if p is not None}
    if len(dev) > 1:
        raise ValueError("output buffers must all be host or all device")
    res.flags = DSG_DST_DEVICE if dev == {True} else 0
    res.best, res.loads, res.sets, res.trace = pb, pl, ps, pt
    _check(ctx, LIB.dsg_run_batch(batch, variant, T.ctypes.data,
                                  None if en is None else en.ctypes.data,
                                  None if ed is None else ed.ctypes.data,
                                  threads_per_graph, ctypes.byref(res)))


def dsg_set_batch_tuning(ctx, batch, thread_degree: int = 0, block_degree: int = 0) -> None:
    """Tuning of later dsg_run_batch calls (0 = default): thread-vs-warp list
    length of the PaRSorting++ scan, whole-block degree of the PaRGreedy++ rounds."""
    _check(ctx, LIB.dsg_set_batch_tuning(batch, thread_degree, block_degree))


def dsg_free_batch(batch) -> None:
    LIB.dsg_free_batch(batch)


def dsg_server_create(device: int = 0, slots: int = 4, hbm_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    rc = LIB.dsg_server_create(device, slots, hbm_budget_bytes, ctypes.byref(out))
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_server_create")
    return out.value


def dsg_server_submit(server, n: int, offsets, adj, variant: int, T: int, eps_num: int = 0,
                      eps_den: int = 1) -> int:
    po, _ = _ptr(offsets, np.int64)
    pa, _ = _ptr(adj, np.int32)
    _need(offsets, max(int(n), 0) + 1, "offsets")
    if n >= 0:
        _need(adj, int(offsets[n]), "adj")
    t = ctypes.c_uint64(0)
    rc = LIB.dsg_server_submit(server, n, po, pa, variant, T, eps_num, eps_den, ctypes.byref(t))
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_server_submit")
    return t.value


def dsg_server_wait(server, ticket: int, timeout_ms: int = -1, loads=None, best_set=None) -> dict | None:
    """Result dict, or None if the request is not finished within timeout_ms."""
    res = dsg_server_result()
    pl, _ = _ptr(loads, np.int64)
    ps, _ = _ptr(best_set, np.int32)
    rc = LIB.dsg_server_wait(server, ticket, timeout_ms, ctypes.byref(res), pl, ps)
    if rc == DSG_ERR_BUSY:
        return None
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_server_wait")
    return {f: (getattr(res, f).decode() if f == "error" else getattr(res, f))
            for f, _ in dsg_server_result._fields_}


def dsg_server_stats(server) -> dict:
    v = [ctypes.c_int64() for _ in range(5)]
    rc = LIB.dsg_server_stats(server, *[ctypes.byref(x) for x in v])
    if rc != DSG_OK:
        raise DsgError(rc, "dsg_server_stats")
    return dict(zip(["queued", "running", "done", "bytes_in_use", "budget"], [x.value for x in v]))


def dsg_server_destroy(server) -> None:
    LIB.dsg_server_destroy(server)


DSG_NOALLOC_MAX_VERTICES = 262144

EXPORTED = ["dsg_create", "dsg_destroy", "dsg_last_error", "dsg_debug_set", "dsg_upload_csr", "dsg_graph_info",
            "dsg_run", "dsg_free_graph", "dsg_set_profiling", "dsg_get_stats", "dsg_get_peel_stats",
            "dsg_densest_suffix_noalloc", "dsg_upload_batch", "dsg_batch_info", "dsg_run_batch",
            "dsg_set_batch_tuning", "dsg_free_batch", "dsg_coreness", "dsg_apx_coreness", "dsg_run_pruned", "dsg_run_pruned_apx", "dsg_run_pruned_apx_exact", "dsg_server_create", "dsg_server_submit", "dsg_server_wait",
            "dsg_server_stats", "dsg_server_destroy"]
