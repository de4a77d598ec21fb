// batch.h -- device layout of a packed batch of graphs (k_batch.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "internal.h"

namespace dsg {

struct BatchDev {
    int32_t G;
    int32_t Tmax;
    const int64_t *vbase;     // [G+1] first packed vertex of each graph
    const int64_t *off;       // [N+1] global arc index of each vertex's list
    const int32_t *adj;       // [arcs] local ids
    const int32_t *order;     // [G] processing order (largest graph first)
    const int32_t *T;         // [G] iterations per graph
    const int64_t *pq;        // [2G] eps = pq[2g] / pq[2g+1] (PaRGreedy++)
    const int64_t *init;      // [N] initial loads or nullptr
    uint32_t *loads;          // [N]
    uint32_t *A;              // [N]
    uint32_t *keys;           // [2N]
    uint32_t *ids;            // [2N]
    uint32_t *best_loads;     // [N] loads (PaRSorting++) or rounds (PaRGreedy++) of the best iteration
    uint32_t *round;          // [N] PaRGreedy++ round of each vertex
    int64_t *loads_out;       // [N] or nullptr
    int32_t *sets;            // [N] or nullptr (graph g's set at vbase[g])
    int64_t *best;            // [G][4]: edges, vertices, iteration, set size
    int64_t *trace;           // [G][Tmax][3] or nullptr
    // tuning knobs (dsg_set_batch_tuning): lists shorter than thread_deg arcs
    // are scanned by one thread, longer ones by a warp (PaRSorting++); F
    // vertices above block_deg arcs are counted by the whole block (PaRGreedy++)
    int32_t thread_deg = 32;
    int32_t block_deg = 1024;
};

cudaError_t launch_batch_validate(const BatchDev &B, int full, int32_t *err, cudaStream_t s);
// variant: DSG_SORTING or DSG_PEELING
cudaError_t launch_batch(const BatchDev &B, int variant, int threads, int sm_count, uint32_t *graph_ctr,
                         cudaStream_t s);

}  // namespace dsg
