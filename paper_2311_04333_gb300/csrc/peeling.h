// peeling.h -- host side of the PaRGreedy++ round peel (k_peeling.cu).
#pragma once
#include <string>
#include "internal.h"

struct dsg_ctx;

namespace dsg {

struct PeelBufs {
    void *mem = nullptr;
    size_t bytes = 0;
};

void peel_free(PeelBufs &pb, cudaStream_t s);

// Caps the PaRGreedy++ grid of runs on ctx (0: one block per SM).  Grids
// whose sizes add up to at most the SM count are co-resident together: each
// peel block needs an SM of its own, and nothing else waits on them.
void ctx_set_peel_max_blocks(dsg_ctx *ctx, int blocks);

// Scratch of kcore_run, reused across calls on graphs up to its size.
struct KCoreBufs {
    void *mem = nullptr;
    size_t bytes = 0;
    ~KCoreBufs();
};
// The k-core of g by deletion: keep[v] = k for its vertices, 0 for the
// others; *survivors = its size.  ctl receives bounded-wait errors.
int kcore_run(cudaStream_t s, const GraphDev &g, Control *ctl, int sm_count, KCoreBufs &kb, int32_t k,
              int32_t *keep, int64_t *survivors, std::string &err);
void kcore_free(KCoreBufs &kb, cudaStream_t s);

// Core numbers of g (int32[n]) and their maximum, by the eps = 0 round peel
// from zero loads; ctl only receives bounded-wait errors.
int coreness_run(cudaStream_t s, const GraphDev &g, Control *ctl, int sm_count, int32_t *core, int64_t *kmax,
                 std::string &err);

// Runs T PaRGreedy++ iterations on g with eps = p/q, leaving the same state
// as the sorting path (loads, best in ctl, best_loads snapshot, trace).  The
// cooperative peel uses at most max_blocks blocks (and one per SM at most).
// Returns a dsg_status; *launches counts kernel launches.
int peel_run(cudaStream_t s, const GraphDev &g, RunBufs &b, PeelBufs &pb, bool &pb_ready,
             int sm_count, int max_blocks, int T, int64_t p, int64_t q, int *launches, std::string &err);

}  // namespace dsg
