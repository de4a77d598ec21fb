// graphgen_cuda.cu -- GPU side of the seeded R-MAT recipe (graphgen.h): the
// same counter-based draws as the CPU generator, so both produce the same
// graph.  Two kernels: per-vertex arc counts, and placement of every arc
// into its source's slot range (order within a list is fixed later by a
// sort).  No part of the densest-subgraph method is here.
#include <cstdint>
#include <cuda_runtime.h>
#include "graphgen.h"

namespace {

__global__ void k_count(uint64_t key, int scale, uint64_t E, const uint32_t *xu, const uint32_t *xv,
                        uint64_t nx, uint32_t *deg)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E + nx;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u, v;
        if (i < E) gg_rmat_edge(key, scale, i, &u, &v);
        else { u = xu[i - E]; v = xv[i - E]; }
        if (u == v) continue;
        atomicAdd(&deg[u], 1u);
        atomicAdd(&deg[v], 1u);
    }
}

__global__ void k_fill(uint64_t key, int scale, uint64_t E, const uint32_t *xu, const uint32_t *xv,
                       uint64_t nx, const int64_t *off, uint32_t *cursor, int32_t *adj)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E + nx;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u, v;
        if (i < E) gg_rmat_edge(key, scale, i, &u, &v);
        else { u = xu[i - E]; v = xv[i - E]; }
        if (u == v) continue;
        adj[off[u] + atomicAdd(&cursor[u], 1u)] = (int32_t)v;
        adj[off[v] + atomicAdd(&cursor[v], 1u)] = (int32_t)u;
    }
}

}  // namespace

extern "C" {

// arcs per source vertex (self-loops dropped, duplicates kept); deg must be
// zeroed, n = 2^scale entries.  Returns a cudaError_t.
int gg_cuda_count(uint64_t seed, int scale, uint64_t E, const uint32_t *xu, const uint32_t *xv,
                  uint64_t nx, uint32_t *deg, void *stream)
{
    const uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    k_count<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(key, scale, E, xu, xv, nx, deg);
    return (int)cudaGetLastError();
}

// place every arc at off[src] + cursor[src]++ ; cursor must be zeroed.
int gg_cuda_fill(uint64_t seed, int scale, uint64_t E, const uint32_t *xu, const uint32_t *xv,
                 uint64_t nx, const int64_t *off, uint32_t *cursor, int32_t *adj, void *stream)
{
    const uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    k_fill<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(key, scale, E, xu, xv, nx, off, cursor, adj);
    return (int)cudaGetLastError();
}

}
