// k_prune.cu -- getCore of the Pruning-and-Refining framework (arXiv
// 2311.04333, Alg. 1, initial and re-pruning): the subgraph induced on the vertices
// whose core number (in the input graph) reaches a level, relabelled in
// increasing id so that every list stays in its order, with the maps that
// carry loads and ids across the relabelling.
#include "common.cuh"
#include "prune.h"

namespace dsg {
namespace {

// pos[v] = 1 if v is kept (pos[n] = 0); scanned into new ids afterwards
__global__ void k_ext_flags(const int32_t *__restrict__ core, const int32_t *__restrict__ old_of, int key_local,
                            int64_t n, int64_t level, int64_t *pos)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = 0;
        if (v < n) k = core[(old_of && !key_local) ? old_of[v] : (int32_t)v] >= level ? 1 : 0;
        pos[v] = k;
    }
}

__device__ __forceinline__ bool kept(const int64_t *pos, int64_t v) { return pos[v + 1] != pos[v]; }

// warp per vertex: kept neighbours of each kept vertex
__global__ void k_ext_deg(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int64_t n,
                          const int64_t *__restrict__ pos, int64_t *ndeg)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        if (!kept(pos, v)) continue;
        uint32_t c = 0;
        for (int64_t j = off[v] + lane; j < off[v + 1]; j += 32) c += kept(pos, adj[j]) ? 1u : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) ndeg[pos[v]] = c;
    }
}

// warp per vertex: the kept neighbours' new ids, in list order
__global__ void k_ext_fill(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int64_t n,
                           const int64_t *__restrict__ pos, const int64_t *__restrict__ noff, int32_t *nadj)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < n; v += nw) {
        if (!kept(pos, v)) continue;
        int64_t o = noff[pos[v]];
        for (int64_t j0 = off[v]; j0 < off[v + 1]; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool ok = j < off[v + 1];
            const int32_t w = ok ? adj[j] : 0;
            const bool k = ok && kept(pos, w);
            const uint32_t m = __ballot_sync(0xffffffffu, k);
            if (k) nadj[o + __popc(m & lanemask_lt())] = (int32_t)pos[w];
            o += __popc(m);
        }
    }
}

// ids and loads across the relabelling; loads of dropped vertices are
// written to frozen[] at their original ids
__global__ void k_ext_map(int64_t n, const int64_t *__restrict__ pos, const int32_t *__restrict__ old_of,
                          const int64_t *__restrict__ loads, int32_t *nold, int64_t *nloads, int64_t *frozen)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = old_of ? old_of[v] : (int32_t)v;
        const int64_t l = loads ? loads[v] : 0;
        if (kept(pos, v)) {
            nold[pos[v]] = o;
            nloads[pos[v]] = l;
        } else if (frozen) {
            frozen[o] = l;
        }
    }
}

__global__ void k_gather_ids(const int32_t *__restrict__ local, int64_t k, const int32_t *__restrict__ old_of,
                             int32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = old_of[local[i]];
}

__global__ void k_scatter_loads(const int64_t *__restrict__ loads, int64_t n, const int32_t *__restrict__ old_of,
                                int64_t *out)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[old_of[v]] = loads[v];
}

// degrees as int32
__global__ void k_deg32(const int64_t *__restrict__ off, int64_t n, int32_t *deg)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        deg[v] = (int32_t)(off[v + 1] - off[v]);
}

__device__ __forceinline__ int ilog2(uint32_t x) { return 31 - __clz(x); }

// warp per vertex: vertices by floor(log2 degree), edges {u, w} (u < w) by
// floor(log2 min(deg u, deg w))
__global__ void k_minlog_hist(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                              const int32_t *__restrict__ deg, int64_t n, unsigned long long *vh,
                              unsigned long long *eh)
{
    __shared__ unsigned long long sv[32], se[32];
    if (threadIdx.x < 32) {
        sv[threadIdx.x] = 0;
        se[threadIdx.x] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {
        const int32_t du = deg[u];
        if (du == 0) continue;
        if (lane == 0) atomicAdd(&sv[ilog2((uint32_t)du)], 1ull);
        for (int64_t j0 = off[u]; j0 < off[u + 1]; j0 += 32) {
            const int64_t j = j0 + lane;
            int b = 32;                               // no edge
            if (j < off[u + 1]) {
                const int32_t w = adj[j];
                if (w > u) b = ilog2((uint32_t)min(du, deg[w]));
            }
            // one shared-memory add per distinct bin of the warp
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (b < 32 && (peers & lanemask_lt()) == 0) atomicAdd(&se[b], (unsigned long long)__popc(peers));
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        if (sv[threadIdx.x]) atomicAdd(&vh[threadIdx.x], sv[threadIdx.x]);
        if (se[threadIdx.x]) atomicAdd(&eh[threadIdx.x], se[threadIdx.x]);
    }
}

// the same histograms from the degree-oriented copy: an edge is stored at
// its endpoint of smaller (degree, id), so the smaller degree of an edge is
// the degree of the vertex holding it, and no arc is read
__global__ void k_minlog_oriented(const int64_t *__restrict__ off, const int64_t *__restrict__ ooff, int64_t n,
                                  unsigned long long *vh, unsigned long long *eh)
{
    __shared__ unsigned long long sv[32], se[32];
    if (threadIdx.x < 32) {
        sv[threadIdx.x] = 0;
        se[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = off[u + 1] - off[u];
        if (d == 0) continue;
        const int b = ilog2((uint32_t)d);
        atomicAdd(&sv[b], 1ull);
        const int64_t od = ooff[u + 1] - ooff[u];
        if (od) atomicAdd(&se[b], (unsigned long long)od);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        if (sv[threadIdx.x]) atomicAdd(&vh[threadIdx.x], sv[threadIdx.x]);
        if (se[threadIdx.x]) atomicAdd(&eh[threadIdx.x], se[threadIdx.x]);
    }
}

}  // namespace

cudaError_t degree_core_bound(cudaStream_t s, const GraphDev &g, int32_t *deg, int64_t *k_low)
{
    const int64_t n = g.n;
    cudaError_t e;
    DevAllocs A(s);
    unsigned long long *h = nullptr;
    if ((e = A.get(&h, 64 * 8)) != cudaSuccess) return e;
    cudaMemsetAsync(h, 0, 64 * 8, s);
    const int grid = (int)imin64((n + 255) / 256, 152 * 16);
    const int wgrid = (int)imin64((n * 32 + 255) / 256, 152 * 32);
    k_deg32<<<grid, 256, 0, s>>>(g.off, n, deg);
    if (g.ooff) k_minlog_oriented<<<grid, 256, 0, s>>>(g.off, g.ooff, n, h, h + 32);
    else k_minlog_hist<<<wgrid, 256, 0, s>>>(g.off, g.adj, deg, n, h, h + 32);
    unsigned long long hh[64];
    cudaMemcpyAsync(hh, h, sizeof hh, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    // densest of the subgraphs G[deg >= 2^j]: a lower bound on rho*
    int64_t be = 0, bv = 1;
    unsigned long long V = 0, E = 0;
    for (int j = 31; j >= 0; --j) {
        V += hh[j];
        E += hh[32 + j];
        if (V > 0 && (__int128)E * bv > (__int128)be * (__int128)V) {
            be = (int64_t)E;
            bv = (int64_t)V;
        }
    }
    const int64_t ceil_rho = (be + bv - 1) / bv;
    *k_low = (ceil_rho + 1) / 2;
    return cudaGetLastError();
}

cudaError_t extract_core(cudaStream_t s, int64_t n, const int64_t *off, const int32_t *adj, const int32_t *core,
                         const int32_t *old_of, int64_t level, const int64_t *loads, int64_t *frozen, CoreGraph *out,
                         bool key_local)
{
    cudaError_t e;
    DevAllocs A(s);
    int64_t *pos = nullptr, *tmp = nullptr;
    const int64_t ntmp = scan_tmp_count(n + 1) + 2;
    if ((e = A.get(&pos, 8 * (size_t)(n + 1))) != cudaSuccess) return e;
    if ((e = A.get(&tmp, 8 * (size_t)ntmp)) != cudaSuccess) return e;
    int64_t *total = tmp + ntmp - 1;
    const int grid = (int)imin64((n + 256) / 256, 152 * 16);
    const int wgrid = (int)imin64((n * 32 + 255) / 256, 152 * 32);
    k_ext_flags<<<grid, 256, 0, s>>>(core, old_of, key_local ? 1 : 0, n, level, pos);
    if ((e = scan_exclusive_i64(pos, n + 1, total, tmp, s)) != cudaSuccess) return e;
    int64_t nn = 0;
    cudaMemcpyAsync(&nn, total, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    int64_t *noff = nullptr, *nloads = nullptr;
    int32_t *nold = nullptr, *nadj = nullptr;
    if ((e = A.get(&noff, 8 * (size_t)(nn + 1))) != cudaSuccess ||
        (e = A.get(&nold, 4 * (size_t)imax64(nn, 1))) != cudaSuccess ||
        (e = A.get(&nloads, 8 * (size_t)imax64(nn, 1))) != cudaSuccess)
        return e;
    cudaMemsetAsync(noff, 0, 8 * (size_t)(nn + 1), s);
    k_ext_deg<<<wgrid, 256, 0, s>>>(off, adj, n, pos, noff);
    if ((e = scan_exclusive_i64(noff, nn + 1, total, tmp, s)) != cudaSuccess) return e;
    int64_t arcs = 0;
    cudaMemcpyAsync(&arcs, total, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if ((e = A.get(&nadj, 4 * (size_t)imax64(arcs, 1))) != cudaSuccess) return e;
    k_ext_fill<<<wgrid, 256, 0, s>>>(off, adj, n, pos, noff, nadj);
    k_ext_map<<<grid, 256, 0, s>>>(n, pos, old_of, loads, nold, nloads, frozen);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the core's arrays go to the caller; A frees pos and tmp (stream-ordered)
    A.keep(noff);
    A.keep(nadj);
    A.keep(nold);
    A.keep(nloads);
    out->n = nn;
    out->arcs = arcs;
    out->off = noff;
    out->adj = nadj;
    out->old_of = nold;
    out->loads = nloads;
    return cudaSuccess;
}

void free_core(CoreGraph &c, cudaStream_t s)
{
    if (c.off) cudaFreeAsync(c.off, s);
    if (c.adj) cudaFreeAsync(c.adj, s);
    if (c.old_of) cudaFreeAsync(c.old_of, s);
    if (c.loads) cudaFreeAsync(c.loads, s);
    c = CoreGraph{};
}

cudaError_t gather_ids(const int32_t *local, int64_t k, const int32_t *old_of, int32_t *out, cudaStream_t s)
{
    if (k > 0) k_gather_ids<<<(int)imin64((k + 255) / 256, 152 * 8), 256, 0, s>>>(local, k, old_of, out);
    return cudaGetLastError();
}

namespace {
__global__ void k_scatter_ids(const int32_t *__restrict__ x, int64_t n, const int32_t *__restrict__ old_of, int32_t *out)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[old_of[v]] = x[v];
}
}  // namespace

cudaError_t scatter_ids(const int32_t *x, int64_t n, const int32_t *old_of, int32_t *out, cudaStream_t s)
{
    if (n > 0) k_scatter_ids<<<(int)imin64((n + 255) / 256, 152 * 8), 256, 0, s>>>(x, n, old_of, out);
    return cudaGetLastError();
}

namespace {
__global__ void k_assign_removed(const int32_t *__restrict__ keep, int64_t n, const int32_t *__restrict__ old_of,
                                 int32_t value, int32_t *out)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (keep[v] == 0) out[old_of ? old_of[v] : v] = value;
}
}  // namespace

cudaError_t assign_removed(const int32_t *keep, int64_t n, const int32_t *old_of, int32_t value, int32_t *out,
                           cudaStream_t s)
{
    if (n > 0) k_assign_removed<<<(int)imin64((n + 255) / 256, 152 * 8), 256, 0, s>>>(keep, n, old_of, value, out);
    return cudaGetLastError();
}

cudaError_t scatter_loads(const int64_t *loads, int64_t n, const int32_t *old_of, int64_t *out, cudaStream_t s)
{
    if (n > 0) k_scatter_loads<<<(int)imin64((n + 255) / 256, 152 * 8), 256, 0, s>>>(loads, n, old_of, out);
    return cudaGetLastError();
}

}  // namespace dsg
