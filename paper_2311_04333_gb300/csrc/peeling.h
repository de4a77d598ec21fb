// peeling.h -- host side of the PaRGreedy++ round peel (k_peeling.cu).
#pragma once
#include <string>
#include "internal.h"

namespace dsg {

struct PeelBufs {
    void *mem = nullptr;
    size_t bytes = 0;
};

void peel_free(PeelBufs &pb, cudaStream_t s);

// Runs T PaRGreedy++ iterations on g with eps = p/q, leaving the same state
// as the sorting path (loads, best in ctl, best_loads snapshot, trace).
// Returns a dsg_status; *launches counts kernel launches.
int peel_run(cudaStream_t s, const GraphDev &g, RunBufs &b, PeelBufs &pb, bool &pb_ready,
             int sm_count, int T, int64_t p, int64_t q, int *launches, std::string &err);

}  // namespace dsg
