// prune.h -- getCore of the Pruning-and-Refining framework (k_prune.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "internal.h"

namespace dsg {

// A core of the input graph in device memory, relabelled: old_of[local] is
// the input id, loads[local] the carried loads.
struct CoreGraph {
    int64_t n = 0, arcs = 0;
    int64_t *off = nullptr;
    int32_t *adj = nullptr;
    int32_t *old_of = nullptr;
    int64_t *loads = nullptr;
};

// The subgraph of (n, off, adj) induced on {v : core[old_of[v]] >= level}
// (old_of NULL: identity; key_local: core[v] by local id), its maps and
// carried loads (loads NULL: zeros); the loads of the dropped vertices go
// to frozen[old id] (if not NULL).
cudaError_t extract_core(cudaStream_t s, int64_t n, const int64_t *off, const int32_t *adj, const int32_t *core,
                         const int32_t *old_of, int64_t level, const int64_t *loads, int64_t *frozen, CoreGraph *out,
                         bool key_local = false);
void free_core(CoreGraph &c, cudaStream_t s);
// deg[n] = degrees (int32), and k_low = ceil(ceil(rho(X)) / 2) for the
// densest X among the subgraphs induced on {v : deg(v) >= 2^j}: since
// k_max >= ceil(rho*) >= ceil(rho(X)), k_low <= ceil(k_max / 2), and every
// k-core with k >= k_low lies in the subgraph induced on {v : deg(v) >= k_low}.
cudaError_t degree_core_bound(cudaStream_t s, const GraphDev &g, int32_t *deg, int64_t *k_low);
// out[i] = old_of[local[i]]
cudaError_t gather_ids(const int32_t *local, int64_t k, const int32_t *old_of, int32_t *out, cudaStream_t s);
// out[old_of[v]] = x[v]
cudaError_t scatter_ids(const int32_t *x, int64_t n, const int32_t *old_of, int32_t *out, cudaStream_t s);
// out[old_of[v]] = value for every v with keep[v] == 0 (old_of NULL: identity)
cudaError_t assign_removed(const int32_t *keep, int64_t n, const int32_t *old_of, int32_t value, int32_t *out,
                           cudaStream_t s);
// levels of the c-approximate k-core decomposition (c = c_num / c_den > 1):
// tau_0 = 1, tau_{i+1} = ceil(tau_i * c)
inline int64_t apx_next_level(int64_t tau, int64_t c_num, int64_t c_den)
{
    return (tau * c_num + c_den - 1) / c_den;
}
// The core order whose vertices are {v : k-hat(v) >= x}: 1 + the largest
// level below x (level 0 below tau_0), 0 for x <= 0.
inline int64_t apx_order(int64_t x, int64_t c_num, int64_t c_den)
{
    if (x <= 0) return 0;
    int64_t below = 0, tau = 1;
    while (tau < x) {
        below = tau;
        tau = apx_next_level(tau, c_num, c_den);
    }
    return below + 1;
}
// out[old_of[v]] = loads[v]
cudaError_t scatter_loads(const int64_t *loads, int64_t n, const int32_t *old_of, int64_t *out, cudaStream_t s);

}  // namespace dsg
