"""Seeded synthetic graph inputs for the densest-subgraph path.

This module holds no part of the method: only deterministic random numbers
(SplitMix64 used as a counter-based generator, see graphgen.h) and graph
recipes.  It serves both the oracle side and the CUDA side of the tests and
the benchmark.  Graphs are undirected and simple, in CSR form with int64
offsets and int32 ascending adjacency lists.

Recipes (the inputs stand in for the paper's SNAP / WebGraph datasets, which
are not available here):
  * ``er_planted_clique``: G(n, p) with per-pair Bernoulli draws plus a
    clique on k seeded-random vertices (n=2000, p=0.005, k=30, seed 1);
  * ``rmat``: R-MAT (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), unpermuted ids,
    optionally with planted G(s, 1/2) blocks on disjoint seeded vertex sets;
  * ``er_m``: a G(n, M)-style graph with a given average degree;
  * ``chung_lu``: power-law expected degrees (exponent gamma);
  * ``batch_mix``: the 4,096-graph mix of the batched workload.
Zero-degree vertices are dropped and the rest relabelled in increasing
original id (the paper removes zero-degree vertices from all inputs).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lib_handle = None


def build() -> str:
    """Compile the CPU generator into graphgen/_build/libgraphgen.so."""
    os.makedirs(_BUILD, exist_ok=True)
    src = [os.path.join(_HERE, "graphgen.c")]
    deps = src + [os.path.join(_HERE, "graphgen.h")]
    if os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(d) for d in deps):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp] + src)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        i64, u64, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.gg_er_planted_clique.argtypes = [i64, u64, u64, i64, u64, p, p, i64]
        lib.gg_er_planted_clique.restype = i64
        lib.gg_rmat.argtypes = [ctypes.c_int, i64, u64, p, p, i64]
        lib.gg_rmat.restype = i64
        lib.gg_planted_blocks.argtypes = [ctypes.c_int, ctypes.c_int, p, u64, p, p, i64, i64]
        lib.gg_planted_blocks.restype = i64
        lib.gg_er_m.argtypes = [i64, i64, u64, p, p, i64]
        lib.gg_er_m.restype = i64
        lib.gg_weighted_pairs.argtypes = [i64, p, i64, u64, p, p, i64]
        lib.gg_weighted_pairs.restype = i64
        lib.gg_build_csr.argtypes = [i64, i64, p, p, ctypes.c_int, p, p, p, p]
        lib.gg_build_csr.restype = i64
        lib.gg_block_perm.argtypes = [u64, p, p]
        lib.gg_block_perm.restype = None
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """Undirected simple graph in CSR form."""
    n: int
    off: np.ndarray          # int64[n+1]
    adj: np.ndarray          # int32[2m], each list ascending
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.off[-1]) // 2

    @property
    def max_degree(self) -> int:
        return int(np.max(np.diff(self.off))) if self.n else 0


def csr_from_pairs(n_raw: int, eu: np.ndarray, ev: np.ndarray, drop_isolated: bool = True,
                   name: str = "", meta: dict | None = None, want_new_id: bool = False) -> Graph:
    """Symmetrise, deduplicate and drop self-loops (and optionally zero-degree
    vertices) of an undirected pair list; returns the CSR graph."""
    eu = np.ascontiguousarray(eu, dtype=np.uint32)
    ev = np.ascontiguousarray(ev, dtype=np.uint32)
    E = int(eu.shape[0])
    off = np.zeros(n_raw + 1, dtype=np.int64)
    adj = np.zeros(max(2 * E, 1), dtype=np.int32)
    new_id = np.zeros(max(n_raw, 1), dtype=np.int64)
    arcs = ctypes.c_int64(0)
    nk = _lib().gg_build_csr(n_raw, E, _ptr(eu), _ptr(ev), int(drop_isolated), _ptr(off),
                             _ptr(adj), _ptr(new_id), ctypes.addressof(arcs))
    if nk < 0:
        raise MemoryError("gg_build_csr failed")
    meta = dict(meta or {})
    meta.update(n_raw=n_raw, pairs=E)
    if want_new_id:
        meta["new_id"] = new_id[:n_raw].copy()
    return Graph(int(nk), off[: nk + 1].copy(), adj[: arcs.value].copy(), name, meta)


def er_planted_clique(n: int = 2000, p: tuple[int, int] = (5, 1000), k: int = 30, seed: int = 1,
                      drop_isolated: bool = True) -> Graph:
    """G(n, p) per-pair Bernoulli plus a k-clique on seeded-random vertices."""
    exp = n * (n - 1) / 2 * p[0] / p[1]
    cap = int(exp + 10 * math.sqrt(exp + 1) + 100) + k * (k - 1) // 2
    eu = np.zeros(cap, dtype=np.uint32)
    ev = np.zeros(cap, dtype=np.uint32)
    c = _lib().gg_er_planted_clique(n, p[0], p[1], k, seed, _ptr(eu), _ptr(ev), cap)
    if c < 0:
        raise RuntimeError("edge buffer too small")
    return csr_from_pairs(n, eu[:c], ev[:c], drop_isolated,
                          f"er{n}_p{p[0]}/{p[1]}+K{k}_s{seed}", dict(recipe="er_planted_clique"))


def block_sizes(nblocks: int = 10, step: int = 200) -> list[int]:
    return [step * (b + 1) for b in range(nblocks)]


def rmat(scale: int, edge_factor: int = 16, seed: int = 2, blocks: list[int] | None = None,
         drop_isolated: bool = True, want_new_id: bool = False) -> Graph:
    """R-MAT at `scale` with edge_factor * 2^scale generated edges, optionally
    with planted G(s, 1/2) blocks of the given sizes."""
    E = edge_factor << scale
    extra = 0
    if blocks:
        extra = sum(s * (s - 1) // 2 for s in blocks)
        extra = int(extra / 2 + 10 * math.sqrt(extra) + 100)
    cap = E + extra
    eu = np.zeros(cap, dtype=np.uint32)
    ev = np.zeros(cap, dtype=np.uint32)
    lib = _lib()
    c = lib.gg_rmat(scale, E, seed, _ptr(eu), _ptr(ev), cap)
    if blocks:
        sz = np.asarray(blocks, dtype=np.int64)
        c = lib.gg_planted_blocks(scale, len(blocks), _ptr(sz), seed, _ptr(eu), _ptr(ev), c, cap)
        if c < 0:
            raise RuntimeError("edge buffer too small")
    name = f"rmat{scale}_ef{edge_factor}_s{seed}" + (f"+{len(blocks)}blocks" if blocks else "")
    return csr_from_pairs(1 << scale, eu[:c], ev[:c], drop_isolated, name,
                          dict(recipe="rmat", scale=scale, edge_factor=edge_factor,
                               blocks=list(blocks or [])), want_new_id)


_SO_LARGE = os.path.join(_BUILD, "libgraphgen_large.so")
_large_handle = None


def _large_lib():
    """The bucketed CSR builder (rmat_large.c, OpenMP), compiled on first use."""
    global _large_handle
    if _large_handle is None:
        os.makedirs(_BUILD, exist_ok=True)
        src = os.path.join(_HERE, "rmat_large.c")
        deps = [src, os.path.join(_HERE, "graphgen.h")]
        if not (os.path.exists(_SO_LARGE)
                and all(os.path.getmtime(_SO_LARGE) >= os.path.getmtime(d) for d in deps)):
            tmp = _SO_LARGE + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC",
                                   "-o", tmp, src])
            os.replace(tmp, _SO_LARGE)
        lib = ctypes.CDLL(_SO_LARGE)
        i64, u64, u32, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.gg_large_count.argtypes = [ctypes.c_int, i64, u64, p, p, i64, p]
        lib.gg_large_count.restype = None
        lib.gg_large_bucket.argtypes = [ctypes.c_int, i64, u64, p, p, i64, u32, u32, p, p, i64, p, p]
        lib.gg_large_bucket.restype = i64
        _large_handle = lib
    return _large_handle


def rmat_large(scale: int, edge_factor: int = 16, seed: int = 2, blocks: list[int] | None = None,
               bucket_arcs: int = 1 << 30, log=None) -> Graph:
    """The `rmat` recipe (isolated vertices dropped) built bucket by bucket of
    source vertices, so that host memory holds the CSR plus two buffers of
    `bucket_arcs` 64-bit keys instead of the whole pair list: scale 27 fits in
    about 40 GB.  Same graph as `rmat`, which a CPU test checks."""
    lib = _large_lib()
    E = edge_factor << scale
    n_raw = 1 << scale
    if blocks:
        extra = sum(s * (s - 1) // 2 for s in blocks)
        cap = int(extra / 2 + 10 * math.sqrt(extra) + 100)
        xu = np.zeros(cap, dtype=np.uint32)
        xv = np.zeros(cap, dtype=np.uint32)
        sz = np.asarray(blocks, dtype=np.int64)
        nx = _lib().gg_planted_blocks(scale, len(blocks), _ptr(sz), seed, _ptr(xu), _ptr(xv), 0, cap)
        if nx < 0:
            raise RuntimeError("edge buffer too small")
    else:
        nx = 0
        xu = xv = np.zeros(1, dtype=np.uint32)
    cnt = np.zeros(n_raw, dtype=np.uint32)
    lib.gg_large_count(scale, E, seed, _ptr(xu), _ptr(xv), nx, _ptr(cnt))
    csum = np.concatenate([[0], np.cumsum(cnt, dtype=np.int64)])
    raw_arcs = int(csum[-1])
    bucket_arcs = max(min(bucket_arcs, raw_arcs), int(cnt.max(initial=0)), 1)
    del cnt
    adj = np.empty(max(raw_arcs, 1), dtype=np.int32)
    deg = np.zeros(n_raw, dtype=np.int64)
    buf = np.empty(bucket_arcs, dtype=np.uint64)
    tmp = np.empty(bucket_arcs, dtype=np.uint64)
    at, lo = 0, 0
    while lo < n_raw:
        hi = int(np.searchsorted(csum, csum[lo] + bucket_arcs, side="right")) - 1
        hi = max(min(hi, n_raw), lo + 1)
        k = lib.gg_large_bucket(scale, E, seed, _ptr(xu), _ptr(xv), nx, lo, hi, _ptr(buf), _ptr(tmp),
                                bucket_arcs, adj.ctypes.data + 4 * at, deg.ctypes.data + 8 * lo)
        if k < 0:
            raise RuntimeError("bucket buffer too small")
        if log:
            log(f"bucket [{lo}, {hi}): {k} arcs")
        at += k
        lo = hi
    del buf, tmp, csum
    keep = deg > 0
    nid = np.cumsum(keep, dtype=np.int64) - 1
    nid = nid.astype(np.int32)
    step = 1 << 28
    for a in range(0, at, step):
        b = min(a + step, at)
        adj[a:b] = nid[adj[a:b]]
    del nid
    nk = int(keep.sum())
    off = np.zeros(nk + 1, dtype=np.int64)
    np.cumsum(deg[keep], out=off[1:])
    name = f"rmat{scale}_ef{edge_factor}_s{seed}" + (f"+{len(blocks)}blocks" if blocks else "")
    return Graph(nk, off, adj[:at], name,
                 dict(recipe="rmat", scale=scale, edge_factor=edge_factor, blocks=list(blocks or []),
                      n_raw=n_raw, pairs=E + nx))


def block_vertices(scale: int, seed: int, blocks: list[int]) -> list[np.ndarray]:
    """Raw (pre-relabel) vertex ids of each planted block."""
    mul = ctypes.c_uint64(0)
    add = ctypes.c_uint64(0)
    _lib().gg_block_perm(seed, ctypes.addressof(mul), ctypes.addressof(add))
    mask = (1 << scale) - 1
    out, base = [], 0
    for s in blocks:
        xs = np.arange(base, base + s, dtype=np.uint64)
        out.append(((xs * np.uint64(mul.value) + np.uint64(add.value)) & np.uint64(mask)).astype(np.int64))
        base += s
    return out


def er_m(n: int, avg_degree: float, seed: int, drop_isolated: bool = True) -> Graph:
    """Random graph with about n*avg_degree/2 edge draws (G(n, M) style)."""
    M = max(1, int(round(n * avg_degree / 2)))
    eu = np.zeros(M, dtype=np.uint32)
    ev = np.zeros(M, dtype=np.uint32)
    _lib().gg_er_m(n, M, seed, _ptr(eu), _ptr(ev), M)
    return csr_from_pairs(n, eu, ev, drop_isolated, f"erm{n}_d{avg_degree:g}_s{seed}",
                          dict(recipe="er_m"))


def chung_lu(n: int, avg_degree: float, gamma: float, seed: int, drop_isolated: bool = True) -> Graph:
    """Chung-Lu power-law graph: endpoint i drawn with probability proportional
    to w_i = (i + 1)^(-1/(gamma - 1)) (integer weights, scaled by 2^20)."""
    M = max(1, int(round(n * avg_degree / 2)))
    w = np.floor((np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))) * (1 << 20)) + 1
    cum = np.cumsum(w.astype(np.uint64)).astype(np.uint64)
    eu = np.zeros(M, dtype=np.uint32)
    ev = np.zeros(M, dtype=np.uint32)
    _lib().gg_weighted_pairs(n, _ptr(cum), M, seed, _ptr(eu), _ptr(ev), M)
    return csr_from_pairs(n, eu, ev, drop_isolated, f"cl{n}_d{avg_degree:g}_g{gamma:g}_s{seed}",
                          dict(recipe="chung_lu"))


def _batch_one(args):
    g, seed, n_lo, n_hi = args
    return _batch_graph(g, seed, n_lo, n_hi)


def batch_mix(G: int = 4096, seed: int = 4, n_lo: int = 50, n_hi: int = 50000,
              processes: int = 1) -> list[Graph]:
    """The batched workload (see _batch_graph); `processes` > 1 generates the
    graphs in a spawn-started process pool (safe after CUDA is initialised)."""
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_batch_one, [(g, seed, n_lo, n_hi) for g in range(G)], chunksize=16)
    return [_batch_graph(g, seed, n_lo, n_hi) for g in range(G)]


def _batch_graph(g: int, seed: int, n_lo: int, n_hi: int) -> Graph:
    """The batched workload: n = floor(exp(U(ln n_lo, ln n_hi))); type by index
    mod 3: ER with average degree U[4, 32]; R-MAT at scale ceil(log2 n) with
    edge factor 8 restricted to ids < n; ER with average degree 8 plus a
    planted clique of ceil(2 sqrt(n)) vertices.  Draws come from SplitMix64
    stream 100 of the seed (n) and stream 101 (degree)."""
    u = _py_draw(seed, 100, g) / 2.0**64
    n = int(math.floor(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    n = max(n_lo, min(n_hi, n))
    kind = g % 3
    gseed = seed * 1_000_003 + g
    if kind == 0:
        d = 4 + 28 * (_py_draw(seed, 101, g) / 2.0**64)
        gr = er_m(n, d, gseed, drop_isolated=True)
    elif kind == 1:
        sc = max(1, math.ceil(math.log2(n)))
        E = 8 * n
        eu = np.zeros(E * 2, dtype=np.uint32)
        ev = np.zeros(E * 2, dtype=np.uint32)
        lib = _lib()
        c = lib.gg_rmat(sc, 2 * E, gseed, _ptr(eu), _ptr(ev), 2 * E)
        keep = (eu[:c] < n) & (ev[:c] < n)
        eu2, ev2 = eu[:c][keep][:E], ev[:c][keep][:E]
        gr = csr_from_pairs(n, eu2, ev2, True, f"rmatb{n}_s{gseed}", dict(recipe="rmat_batch"))
    else:
        k = int(math.ceil(2 * math.sqrt(n)))
        M = n * 4
        eu = np.zeros(M + k * (k - 1) // 2, dtype=np.uint32)
        ev = np.zeros_like(eu)
        lib = _lib()
        lib.gg_er_m(n, M, gseed, _ptr(eu), _ptr(ev), M)
        kk = np.array(_py_sample(gseed, n, k), dtype=np.uint32)
        ia, ib = np.triu_indices(k, 1)
        eu[M:] = kk[ia]
        ev[M:] = kk[ib]
        gr = csr_from_pairs(n, eu, ev, True, f"erk{n}_s{gseed}", dict(recipe="er_clique"))
    gr.meta["index"] = g
    return gr


# small deterministic graphs (closed-form test inputs)

def from_edges(n: int, edges, drop_isolated: bool = False, name: str = "") -> Graph:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_pairs(n, e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32),
                          drop_isolated, name)


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], name=f"K{n}")


def star(s: int) -> Graph:
    return from_edges(s + 1, [(0, j) for j in range(1, s + 1)], name=f"star{s}")


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name=f"P{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], name=f"C{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], name=f"K{a},{b}")


def disjoint_union(*gs: Graph) -> Graph:
    edges, base = [], 0
    for g in gs:
        for u in range(g.n):
            for w in g.adj[g.off[u]:g.off[u + 1]]:
                if w > u:
                    edges.append((base + u, base + int(w)))
        base += g.n
    return from_edges(base, edges, name="+".join(g.name for g in gs))


_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _py_key(seed: int, stream: int) -> int:
    return _mix64(((seed * _GOLDEN) & _M64) ^ _mix64(stream + _GOLDEN))


def _py_draw(seed: int, stream: int, i: int) -> int:
    """Draw i of stream `stream` of `seed` (same definition as graphgen.h)."""
    return _mix64(_py_key(seed, stream) + (i + 1) * _GOLDEN)


def _py_sample(seed: int, n: int, k: int) -> list[int]:
    """k distinct ids of 0..n-1 by a partial Fisher-Yates shuffle."""
    perm = list(range(n))
    for i in range(min(k, n)):
        j = i + _py_draw(seed, 102, i) % (n - i)
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:k]


# ---------------------------------------------------------------- GPU generator

_SO_CUDA = os.path.join(_BUILD, "libgraphgen_cuda.so")
_cuda_handle = None


def build_cuda() -> str:
    """Compile the GPU R-MAT generator (nvcc, sm_103a) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "graphgen_cuda.cu")
    deps = [src, os.path.join(_HERE, "graphgen.h")]
    if os.path.exists(_SO_CUDA) and all(os.path.getmtime(_SO_CUDA) >= os.path.getmtime(d) for d in deps):
        return _SO_CUDA
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    tmp = _SO_CUDA + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                           "-Xcompiler", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _SO_CUDA)
    return _SO_CUDA


def _cuda_lib():
    global _cuda_handle
    if _cuda_handle is None:
        lib = ctypes.CDLL(build_cuda())
        u64, p, i = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        lib.gg_cuda_count.argtypes = [u64, i, u64, p, p, u64, p, p]
        lib.gg_cuda_fill.argtypes = [u64, i, u64, p, p, u64, p, p, p, p]
        _cuda_handle = lib
    return _cuda_handle


def rmat_cuda(scale: int, edge_factor: int = 16, seed: int = 2, blocks: list[int] | None = None,
              chunk_arcs: int = 1 << 29):
    """The `rmat` recipe generated on the current CUDA device.  Returns
    (n, off, adj) with off int64[n+1] and adj int32[2m] torch tensors on the
    device; the CSR equals the one `rmat` builds on the CPU."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream().cuda_stream
    lib = _cuda_lib()
    E = edge_factor << scale
    n_raw = 1 << scale
    if blocks:
        extra = sum(s * (s - 1) // 2 for s in blocks)
        cap = int(extra / 2 + 10 * math.sqrt(extra) + 100)
        eu = np.zeros(cap, dtype=np.uint32)
        ev = np.zeros(cap, dtype=np.uint32)
        sz = np.asarray(blocks, dtype=np.int64)
        c = _lib().gg_planted_blocks(scale, len(blocks), _ptr(sz), seed, _ptr(eu), _ptr(ev), 0, cap)
        if c < 0:
            raise RuntimeError("edge buffer too small")
        xu = torch.from_numpy(eu[:c].view(np.int32)).to(dev)
        xv = torch.from_numpy(ev[:c].view(np.int32)).to(dev)
    else:
        c = 0
        xu = xv = torch.zeros(1, dtype=torch.int32, device=dev)
    deg = torch.zeros(n_raw, dtype=torch.int32, device=dev)
    if lib.gg_cuda_count(seed, scale, E, xu.data_ptr(), xv.data_ptr(), c, deg.data_ptr(), stream):
        raise RuntimeError("gg_cuda_count failed")
    off = torch.zeros(n_raw + 1, dtype=torch.int64, device=dev)
    torch.cumsum(deg, 0, out=off[1:])
    arcs_raw = int(off[-1].item())
    adj_raw = torch.empty(max(arcs_raw, 1), dtype=torch.int32, device=dev)
    cursor = torch.zeros(n_raw, dtype=torch.int32, device=dev)
    if lib.gg_cuda_fill(seed, scale, E, xu.data_ptr(), xv.data_ptr(), c, off.data_ptr(),
                        cursor.data_ptr(), adj_raw.data_ptr(), stream):
        raise RuntimeError("gg_cuda_fill failed")
    del cursor, xu, xv
    # sort and deduplicate each list, vertex ranges of at most chunk_arcs arcs
    new_deg = torch.zeros(n_raw, dtype=torch.int64, device=dev)
    off_h = off.cpu().numpy()
    pieces = []
    lo = 0
    while lo < n_raw:
        hi = int(np.searchsorted(off_h, off_h[lo] + chunk_arcs, side="right")) - 1
        hi = max(min(hi, n_raw), lo + 1)
        a, b = int(off_h[lo]), int(off_h[hi])
        if b > a:
            seg = adj_raw[a:b].long()
            src = torch.repeat_interleave(torch.arange(hi - lo, device=dev), deg[lo:hi].long())
            keys = torch.sort((src << 32) | seg).values
            del seg, src
            keep = torch.ones_like(keys, dtype=torch.bool)
            keep[1:] = keys[1:] != keys[:-1]
            keys = keys[keep]
            del keep
            new_deg[lo:hi] = torch.bincount(keys >> 32, minlength=hi - lo)
            pieces.append((keys & 0xFFFFFFFF).to(torch.int32))
            del keys
        lo = hi
    del adj_raw, deg
    adj = torch.cat(pieces) if pieces else torch.zeros(1, dtype=torch.int32, device=dev)
    del pieces
    keepv = new_deg > 0
    newid = torch.cumsum(keepv, 0) - 1
    for a in range(0, adj.numel(), chunk_arcs):
        b = min(a + chunk_arcs, adj.numel())
        adj[a:b] = newid[adj[a:b].long()].to(torch.int32)
    n = int(keepv.sum().item())
    off_new = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(new_deg[keepv], 0, out=off_new[1:])
    m2 = int(off_new[-1].item())
    torch.cuda.synchronize()
    return n, off_new, adj[:m2]
