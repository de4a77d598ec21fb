/*
 * dsg.h -- C ABI of libdsg, the GB300 (sm_103a) implementation of the
 * per-iteration load-weighted peeling of Greedy++ in its two parallel forms
 * (arXiv 2311.04333, "Practical Parallel Algorithms for Near-Optimal
 * Densest Subgraphs on Massive Graphs"):
 *
 *   DSG_SORTING  PaRSorting++ refine step (Sec. 3.2 "GreedySorting++" and
 *                Sec. 3.3 "ParallelGreedySorting++"): each iteration orders
 *                the vertices by their load at the start of the iteration
 *                (ties by vertex id), gives every vertex the number of its
 *                neighbours later in the order (Alg. 3, counts), adds it
 *                to its load (Alg. 3, load update) and takes the densest suffix
 *                of the order (Alg. 3, suffix densities).
 *   DSG_PEELING  PaRGreedy++ refine step (Sec. 3.3 "ParallelGreedy++"): the
 *                order comes from bucketed peeling by l(v) + deg_H(v); each
 *                round peels every alive vertex whose key is within a factor
 *                (1 + p/q) of the minimum key, in ascending id, and applies
 *                the degree decrements at the end of the round.
 *
 * No pruning (Alg. 1) is applied: the refine step runs on the given graph.
 * The problem (Sec. 2): given an undirected unweighted graph G = (V, E),
 * find S maximising |E(S)| / |V(S)|.  All arithmetic is exact integer;
 * densities are returned as (edges, vertices) pairs.
 *
 * Conventions:
 *   - every call returns a dsg_status; no C++ exception crosses the ABI;
 *     dsg_last_error(ctx) describes the last failure on that context;
 *   - uploads COPY the caller's arrays into library-owned device memory;
 *     the caller may free or reuse its buffers as soon as the call returns;
 *   - result buffers are owned by the caller;
 *   - all device work is ordered on the context's CUDA stream; dsg_run and
 *     dsg_run_batch synchronise that stream before they return;
 *   - a context is not thread-safe: use one context per host thread.
 */
#ifndef DSG_H
#define DSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dsg_ctx dsg_ctx;
typedef struct dsg_graph dsg_graph;
typedef struct dsg_batch dsg_batch;

typedef enum {
    DSG_OK = 0,
    DSG_ERR_INVALID = 1,   /* malformed argument or graph */
    DSG_ERR_NOMEM = 2,     /* device or host allocation failed */
    DSG_ERR_CUDA = 3,      /* a CUDA call failed (context may be unusable) */
    DSG_ERR_OVERFLOW = 4,  /* loads or sizes would exceed the device types */
    DSG_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    DSG_ERR_BUSY = 6       /* resource in use (e.g. serving slots full) */
} dsg_status;

typedef enum {
    DSG_SORTING = 0,       /* PaRSorting++ refine step */
    DSG_PEELING = 1        /* PaRGreedy++ refine step, eps = p/q */
} dsg_variant;

/* dsg_upload_csr / dsg_upload_batch flags */
#define DSG_VALIDATE   0x1u  /* check symmetry, no self-loops, no duplicates */
#define DSG_SRC_DEVICE 0x2u  /* offsets/adj are device pointers (else host) */

/* dsg_result.flags */
#define DSG_DST_DEVICE  0x1u /* loads/best_set/trace are device pointers */
#define DSG_INIT_DEVICE 0x2u /* init_loads (dsg_run) is a device pointer */
#define DSG_PATH_GRID   0x4u /* dsg_run: whole-GPU kernels whatever the graph's size */
#define DSG_PATH_BLOCK  0x8u /* dsg_run: one thread block carries all T iterations
                                (default up to 16,384 vertices and 2^19 arcs for
                                DSG_PEELING, 16,384 vertices and 2^18 arcs for
                                DSG_SORTING; the two PATH flags are exclusive) */

/* Output of one run.  The caller sets `flags` and the three buffer
 * pointers (each may be NULL to skip that output); the library fills the
 * scalar fields.
 *   best_edges/best_vertices: |E(S)| and |V(S)| of the best subgraph found
 *     (S = G initially, replaced only by a strictly denser suffix; ties keep
 *     the earliest iteration and, within it, the largest suffix);
 *   best_iter: iteration (1..T) that produced S, 0 if S = G was never beaten;
 *   best_set_size: |V(S)|;
 *   loads[n]: the loads after the last iteration (int64);
 *   best_set[n]: the ids of S in ascending order (first best_set_size used);
 *   trace[3*T]: per iteration t (0-based row t), the densest suffix of that
 *     iteration alone (edges, vertices; largest suffix on ties) and its width
 *     max_v deg*(v) (the per-iteration load increase bound, Sec. 4.4).   */
typedef struct {
    uint32_t flags;
    int32_t best_iter;
    int64_t best_edges;
    int64_t best_vertices;
    int64_t best_set_size;
    int64_t *loads;
    int32_t *best_set;
    int64_t *trace;
} dsg_result;

/* Create a context on CUDA device `device`, issuing all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream is borrowed, not owned.  A context serves one host thread at a
 * time: calls on the same context are not synchronised with one another
 * (the server below gives each of its workers a context of its own).
 * Returns DSG_ERR_CUDA if the device cannot be used and DSG_ERR_INVALID if
 * the library was not built for it. */
int dsg_create(int device, void *cuda_stream, dsg_ctx **out);

/* Release a context.  Graphs and batches created on it must be freed first.
 * Device memory comes from the device's default stream-ordered pool, which
 * the library sets to keep freed blocks cached for reuse; this call returns
 * the unused cached memory to the driver. */
void dsg_destroy(dsg_ctx *ctx);

/* Text of the last error on `ctx` ("" if none).  Valid until the next call
 * on the same context. */
const char *dsg_last_error(const dsg_ctx *ctx);

/* ---- test-only fault hooks ---------------------------------------------- */

/* Knobs that make the library's failure paths run, for tests of failure
 * detection (the paper has no counterpart: its failures are not modelled).
 * All are off by default and cost nothing when off.
 *   DSG_DEBUG_SPIN_LIMIT (ctx): polls before a bounded device-side wait (the
 *     radix passes' look-back, the PaRGreedy++ grid barrier) gives up, for
 *     later dsg_run calls on ctx; 0 restores the default (about a second);
 *   DSG_DEBUG_STALL (ctx): 1 makes tile 0 of every radix pass withhold its
 *     look-back words, 2 keeps block 1 of the PaRGreedy++ round kernel from
 *     arriving at its first grid barrier (graphs of 8,192 or more vertices),
 *     in later dsg_run calls on ctx that take the whole-GPU path; the waits
 *     on what is withheld then run out after the spin limit, the run
 *     returns DSG_ERR_TIMEOUT and the context and graph stay usable; 0 turns
 *     it off;
 *   DSG_DEBUG_FAIL_ALLOC (process-wide, ctx may be NULL): the value-th
 *     memory allocation the library makes from now on (device memory, or
 *     the host context of dsg_create) fails as if memory were exhausted,
 *     so the call that made it returns DSG_ERR_NOMEM; 0 turns it off;
 *   DSG_DEBUG_FAIL_UPLOAD (process-wide, ctx may be NULL): the value-th
 *     host-to-device copy of dsg_upload_csr / dsg_upload_batch from now on
 *     fails and that call returns DSG_ERR_CUDA; 0 turns it off;
 *   DSG_DEBUG_PEEL_BLOCKS (ctx): the whole-GPU PaRGreedy++ round kernel of
 *     later runs on ctx uses at most this many SMs' worth of blocks (two
 *     blocks per SM; the cap each server slot sets on its own context;
 *     results do not depend on it); 0 = every SM.
 * The environment variable DSG_FAULT ("alloc:N", "upload:N", or both
 * separated by a comma), read when the library is loaded, sets the two
 * process-wide countdowns the same way.  Returns DSG_ERR_INVALID for an
 * unknown knob, a value out of range, or a NULL ctx where one is needed. */
typedef enum {
    DSG_DEBUG_SPIN_LIMIT = 1,
    DSG_DEBUG_STALL = 2,
    DSG_DEBUG_FAIL_ALLOC = 3,
    DSG_DEBUG_FAIL_UPLOAD = 4,
    DSG_DEBUG_PEEL_BLOCKS = 5
} dsg_debug_knob;
int dsg_debug_set(dsg_ctx *ctx, int knob, int64_t value);

/* Upload an undirected simple graph in CSR form (Sec. 2: G = (V, E)).
 *   n: number of vertices, 1 <= n < 2^31;
 *   offsets[n+1]: int64, offsets[0] = 0, non-decreasing, offsets[n] = 2m
 *     (each undirected edge appears in both endpoint lists), 2m < 2^40;
 *   adj[2m]: int32 neighbour ids in [0, n).
 * With DSG_VALIDATE the library also checks that every list has no self-loop
 * and no repeated neighbour and that the graph is symmetric; otherwise the
 * caller guarantees it.  Lists need not be sorted.  The graph is copied to
 * device memory; a graph above 32,768 vertices or 2^20 arcs also gets the
 * degree-oriented copy and tile schedule of the whole-GPU edge scan (a
 * smaller one gets them on its first run on the whole-GPU path).
 * flags: DSG_VALIDATE (above); DSG_SRC_DEVICE: offsets and adj are device
 * pointers (copied device to device), otherwise host pointers.  A host graph
 * of at least 2^24 arcs is copied in eight vertex-range chunks on a copy
 * stream of the context while the oriented copy is prepared (pinned host
 * memory lets the copies run asynchronously; pageable memory works, without
 * the overlap).  The call returns after the graph is in place; the caller's
 * arrays may then be freed.
 * Errors: DSG_ERR_INVALID for a malformed graph, DSG_ERR_NOMEM, DSG_ERR_CUDA. */
int dsg_upload_csr(dsg_ctx *ctx, int64_t n, const int64_t *offsets, const int32_t *adj,
                   uint32_t flags, dsg_graph **out);

/* Basic facts about an uploaded graph (any pointer may be NULL). */
int dsg_graph_info(const dsg_graph *g, int64_t *n, int64_t *m, int64_t *max_degree);

/* Run T >= 1 iterations of the refine step `variant` on `g` (Alg. 2 with
 * the ordering of `variant`, the density/load update of Alg. 3).  Both
 * paths (out->flags DSG_PATH_GRID / DSG_PATH_BLOCK, default by size) give
 * identical results.
 *   eps_num/eps_den: eps = p/q for DSG_PEELING (p >= 0, q >= 1, p+q < 2^31);
 *     ignored by DSG_SORTING;
 *   init_loads[n]: loads before iteration 1 (NULL: all zero, as Alg. 2
 *     starts); host memory unless out->flags has DSG_INIT_DEVICE.  Passing the
 *     loads of an earlier run resumes it: T1 then T2 iterations give the
 *     loads of T1 + T2 iterations.
 * Loads are kept as 32-bit unsigned integers on the device:
 * DSG_ERR_OVERFLOW if max(init_loads) + T * max_degree >= 2^32.
 * On the whole-GPU path DSG_PEELING is one cooperative launch with up to one
 * block per SM whose blocks wait on one another: do not overlap two such runs
 * on one GPU from different streams (the server of dsg_server_create shares
 * the GPU between its slots safely).
 * Synchronises the context stream before returning. */
int dsg_run(dsg_graph *g, int variant, int32_t T, int64_t eps_num, int64_t eps_den,
            const int64_t *init_loads, dsg_result *out);

/* ---- Pruning-and-Refining framework ----------------------------------- */

/* Core numbers (Sec. 2, Definition of core number) of every vertex of g into
 * core[n] (int32; a device pointer if flags has DSG_DST_DEVICE) and their
 * maximum k_max (may be NULL).  Computed by the round peel with eps = 0 from
 * zero loads: each round removes the alive vertices of minimum induced
 * degree, and a vertex's core number is the largest round minimum up to its
 * round.  Synchronises the context stream. */
int dsg_coreness(dsg_graph *g, int32_t *core, int64_t *k_max, uint32_t flags);

/* What the pruning saw (dsg_run_pruned). */
typedef struct {
    int64_t k_max;                       /* largest core number of g */
    int64_t core_vertices, core_edges;   /* the ceil(k_max/2)-core the refining starts on */
    int64_t final_vertices;              /* vertices of the core it ends on */
    int64_t L_num, L_den;                /* final density lower bound L = L_num / L_den */
} dsg_prune_info;

/* Alg. 1 (Sec. 3, "Pruning-and-Refining Framework") with exact pruning and
 * T iterations of `variant` as the Refine step: core numbers of g (the
 * eps = 0 round peel); L = ceil(k_max / 2); G <- the L-core, S <- G; then T
 * times: one refine iteration on G, its vertices' loads carried over; if its
 * best suffix S' is strictly denser than S: S <- S', L <- max(L, rho(S)),
 * G <- the ceil(L)-core (by the core numbers of g).  The paper's
 * PaRSorting++ / PaRGreedy++ are this with DSG_SORTING / DSG_PEELING.
 * Outputs, in g's ids: best_edges/best_vertices = rho(S), best_iter = the
 * iteration of the last improvement (0: S is the first core itself),
 * best_set[best_set_size] = S ascending; loads[n] = each vertex's load when
 * it left G (0 if never in the first core); trace[3 t ..] = the refine
 * result of iteration t+1 (edges, vertices) and the vertex count of the G
 * it ran on.  out->flags: DSG_DST_DEVICE only (loads start at zero; paths
 * are chosen by size).  info may be NULL.
 * Errors as dsg_run; DSG_ERR_OVERFLOW if T * max_degree >= 2^32. */
int dsg_run_pruned(dsg_graph *g, int variant, int32_t T, int64_t eps_num, int64_t eps_den, dsg_result *out,
                   dsg_prune_info *info);

/* c-approximate core numbers (Sec. 2, "c-Approx k-Core Decomposition":
 * core(v) / c <= k-hat(v) <= c core(v)), c = c_num / c_den with
 * 1 <= c_den < c_num < 2^31.  The decomposition is taken at the geometric
 * levels tau_0 = 1, tau_{i+1} = ceil(tau_i * c): k-hat(v) is the smallest
 * level >= core(v) (0 when core(v) = 0), so core(v) <= k-hat(v) < c core(v).
 * Computed by peeling level by level (the (tau_i + 1)-core of the previous
 * core, by deletion), about log_c(k_max) peels instead of k_max.
 * core[n] (int32) is host memory unless flags has DSG_DST_DEVICE; *k_max
 * (may be NULL) receives the largest k-hat.  Synchronises the context stream.
 * Errors: DSG_ERR_INVALID (c out of range), DSG_ERR_NOMEM, DSG_ERR_CUDA,
 * DSG_ERR_TIMEOUT. */
int dsg_apx_coreness(dsg_graph *g, int64_t c_num, int64_t c_den, int32_t *core, int64_t *k_max, uint32_t flags);

/* Alg. 1 with approximate pruning (Sec. 4, the approximate variants:
 * PaRApxSorting++ with DSG_SORTING; c = 1.5 in the paper's experiments):
 * as dsg_run_pruned, with the core numbers replaced by the c-approximate
 * ones of dsg_apx_coreness, L = ceil(k-hat_max / (2c)) (the corollary on the
 * approximate k_max, which keeps the densest subgraph in the first core),
 * and every getCore keeping {v : k-hat(v) >= ceil(L)}.  Since k-hat >= core,
 * each such set is an exact core (of order 1 + the largest level below
 * ceil(L)); k_max is only bracketed, by about log_c of its range of core
 * tests from the degree bound, instead of located.  info->k_max receives
 * k-hat_max.  Errors as dsg_run_pruned, and DSG_ERR_INVALID for c as in
 * dsg_apx_coreness (c_num = 0 is refused: that is dsg_run_pruned). */
int dsg_run_pruned_apx(dsg_graph *g, int variant, int32_t T, int64_t eps_num, int64_t eps_den, int64_t c_num,
                       int64_t c_den, dsg_result *out, dsg_prune_info *info);

/* Alg. 1 with approximate pruning followed by exact pruning (Sec. 4, the
 * approximate variants: PaRApxGreedy++ with DSG_PEELING).  The c-approximate
 * levels first bracket k_max in (tau_{i-1}, tau_i] with about log_c core tests
 * on shrinking cores, which prunes G to its (tau_{i-1} + 1)-core; k_max is
 * then found exactly inside that bracket by bisection over k-cores of that
 * core, and the run continues as dsg_run_pruned: L = ceil(k_max / 2), exact
 * cores for every getCore.  The outputs equal dsg_run_pruned's (every core
 * the loop takes has order >= ceil(k_max / 2), inside the approximate core);
 * only the work of the set-up differs.  info->k_max receives the exact
 * k_max.  Errors as dsg_run_pruned_apx. */
int dsg_run_pruned_apx_exact(dsg_graph *g, int variant, int32_t T, int64_t eps_num, int64_t eps_den,
                             int64_t c_num, int64_t c_den, dsg_result *out, dsg_prune_info *info);

/* Free an uploaded graph (stream-ordered release of its device memory). */
void dsg_free_graph(dsg_graph *g);

/* ---- batches of small graphs --------------------------------------------- */

/* Per-graph outputs of dsg_run_batch.  The caller sets the pointers (loads,
 * sets and trace may be NULL; best may not) and flags:
 *   best[4*g .. 4*g+3]: best edges, best vertices, best iteration (0 = S = G
 *     never beaten) and best-set size of graph g (the fields of dsg_result);
 *   loads[N]: final loads, graph g's at positions vbase(g) .. vbase(g)+n_g-1
 *     where vbase(g) = n_0 + ... + n_{g-1} (the packing order);
 *   sets[N]: graph g's best set (ascending local ids) from position vbase(g);
 *   trace[3*(g*Tmax + t)]: as dsg_result.trace, Tmax = max_g T[g]. */
typedef struct {
    uint32_t flags;       /* DSG_DST_DEVICE: pointers below are device pointers */
    int64_t *best;
    int64_t *loads;
    int32_t *sets;
    int64_t *trace;
} dsg_batch_result;

/* Upload G >= 1 graphs as one packed batch (copied; host arrays).  Graph g
 * has n_per[g] >= 1 vertices, offsets[g][0..n_per[g]] (int64, starting at 0)
 * and adj[g] (int32 local ids); the same rules as dsg_upload_csr apply to
 * each (DSG_VALIDATE adds the strict-order and symmetry checks).  The total
 * vertex count must stay below 2^31.  Errors: DSG_ERR_INVALID, DSG_ERR_NOMEM. */
int dsg_upload_batch(dsg_ctx *ctx, int32_t G, const int64_t *n_per, const int64_t *const *offsets,
                     const int32_t *const *adj, uint32_t flags, dsg_batch **out);

/* Number of graphs, total vertices and total edges of a batch. */
int dsg_batch_info(const dsg_batch *b, int32_t *G, int64_t *total_n, int64_t *total_m);

/* Run T[g] >= 1 iterations of the refine step `variant` on every graph g of
 * the batch in one persistent launch: each thread block takes whole graphs,
 * largest first, and runs all their iterations (loads start at zero).  The
 * results of graph g are those dsg_run(variant, T[g], eps_num[g],
 * eps_den[g]) gives on it alone.
 *   variant: DSG_SORTING (PaRSorting++) or DSG_PEELING (PaRGreedy++, whose
 *     rounds a block peels by itself with block-wide barriers);
 *   eps_num[G], eps_den[G]: eps = p/q per graph for DSG_PEELING (NULL:
 *     p = 0, q = 1); p >= 0, q >= 1, p + q < 2^31; ignored by DSG_SORTING;
 *   threads_per_graph: 256, 512 or 1024 threads per block, 0 = default
 *     (the tuning knob an autotuner sets).
 * DSG_ERR_OVERFLOW if a graph's T * max_degree reaches 2^32 or p + q
 * reaches 2^31.  Synchronises the context stream before returning. */
int dsg_run_batch(dsg_batch *b, int variant, const int32_t *T, const int64_t *eps_num,
                  const int64_t *eps_den, int32_t threads_per_graph, dsg_batch_result *out);

/* Tuning of later dsg_run_batch calls on b (the knobs an autotuner sets;
 * results do not depend on them):
 *   thread_degree: PaRSorting++ scans lists shorter than this many arcs with
 *     one thread each and longer ones with a warp (0 = default 32, at most
 *     2^20);
 *   block_degree: PaRGreedy++ counts the arcs of a round's peeled vertices
 *     above this degree with the whole block, the others with a warp each
 *     (0 = default 1024, at most 2^30).
 * DSG_ERR_INVALID when a value is out of range. */
int dsg_set_batch_tuning(dsg_batch *b, int32_t thread_degree, int32_t block_degree);

/* Free a batch. */
void dsg_free_batch(dsg_batch *b);

/* ---- serving: continuous batching of requests --------------------------- */

typedef struct dsg_server dsg_server;

/* Outcome of one request (dsg_server_wait). */
typedef struct {
    int32_t status;          /* dsg_status of the request */
    int32_t best_iter;       /* as in dsg_result */
    int64_t best_edges, best_vertices, best_set_size;
    int64_t n, m;
    int32_t slot;            /* worker that ran it (== slots: the batch worker) */
    double queue_ms;         /* submit -> admitted to a slot */
    double run_ms;           /* admitted -> results on the host */
    double latency_ms;       /* submit -> results on the host */
    char error[256];         /* dsg_last_error text when status != DSG_OK */
} dsg_server_result;

/* Start a server on `device` with `slots` workers (1..64), each with its own
 * CUDA stream and context, and an HBM budget in bytes (0 = half the free
 * device memory).  A request is admitted, in arrival order, when a worker is
 * free and its device-memory estimate (about 24m + 128n bytes) fits what the
 * running requests leave of the budget; admitted requests run concurrently
 * on the GPU.  Requests on graphs of at most 32,768 vertices and 2^20 arcs
 * go to one more worker instead, which runs all of them queued at the time
 * it is free as one batch (dsg_run_batch), and so on.  Every request gives
 * exactly what dsg_run gives on it alone. */
int dsg_server_create(int device, int32_t slots, int64_t hbm_budget_bytes, dsg_server **out);

/* Queue one request: a host CSR graph (copied; same rules as dsg_upload_csr),
 * the variant, T and eps = eps_num/eps_den.  *ticket identifies it.
 * DSG_ERR_NOMEM if its estimate exceeds the whole budget, DSG_ERR_INVALID for
 * bad arguments.  The graph itself is checked in full (as with DSG_VALIDATE)
 * when it runs; a bad graph fails its own request only. */
int dsg_server_submit(dsg_server *s, int64_t n, const int64_t *offsets, const int32_t *adj,
                      int variant, int32_t T, int64_t eps_num, int64_t eps_den, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a request; DSG_ERR_BUSY if it is
 * not finished in time.  On return the result is filled (loads[n] and
 * best_set[best_set_size] are copied if the pointers are not NULL) and the
 * ticket is released.  Only one waiter gets a ticket's result: a ticket that
 * is unknown, or that another thread released first, gives DSG_ERR_INVALID. */
int dsg_server_wait(dsg_server *s, uint64_t ticket, int64_t timeout_ms, dsg_server_result *out,
                    int64_t *loads, int32_t *best_set);

/* Queue length, running requests, finished requests, device bytes held by
 * running requests and the budget (any pointer may be NULL). */
int dsg_server_stats(dsg_server *s, int64_t *queued, int64_t *running, int64_t *done,
                     int64_t *bytes_in_use, int64_t *budget);

/* Stop the workers (running requests finish, queued ones are dropped) and
 * free the server.  No other call on this server may be in flight. */
void dsg_server_destroy(dsg_server *s);

/* ---- instrumentation ---------------------------------------------------- */

/* Kernel phases timed when profiling is on (dsg_set_profiling). */
typedef enum {
    DSG_PHASE_EDGE_SCAN = 0,  /* later-neighbour counts (Alg. 3, counts) */
    DSG_PHASE_SORT = 1,       /* radix passes + fused densest suffix */
    DSG_PHASE_OTHER = 2,      /* plan, snapshot, best-set, peeling rounds */
    DSG_PHASE_COUNT = 3
} dsg_phase;

/* Turn per-phase CUDA-event timing on (1) or off (0) for later runs on ctx. */
int dsg_set_profiling(dsg_ctx *ctx, int on);

/* Accumulated statistics since the last reset (reset != 0 clears them):
 *   ms[DSG_PHASE_COUNT]: device milliseconds per phase (profiling on);
 *   launches[DSG_PHASE_COUNT]: kernels launched per phase (always counted);
 *   bytes[DSG_PHASE_COUNT]: algorithmic bytes moved per phase (always). */
int dsg_get_stats(dsg_ctx *ctx, double *ms, int64_t *launches, int64_t *bytes, int reset);

/* PaRGreedy++ telemetry of the whole-GPU dsg_run calls on ctx since the last
 * reset (Sec. 3.3: the rounds of bucketed peeling; the paper's depth bound
 * is in the number of rounds): iterations run, rounds peeled in them, and
 * the alive vertices summed over those rounds (each round touches every
 * alive vertex once).  Any pointer may be NULL; reset != 0 clears them. */
int dsg_get_peel_stats(dsg_ctx *ctx, int64_t *iterations, int64_t *rounds, int64_t *alive_sum, int reset);

/* ---- allocation-free entry point ---------------------------------------- */

/* Largest n accepted by dsg_densest_suffix_noalloc. */
#define DSG_NOALLOC_MAX_VERTICES 262144

/* The densest suffix of the (load, id) order, computed without allocating
 * any memory.  This entry point has no counterpart in the paper; it exists
 * for callers that must not call cudaMalloc: code that runs while a CUDA
 * graph is being captured, code that owns a fixed memory arena and may not
 * grow it (a serving process that reserves its memory at start-up, a plugin
 * living under another framework's allocator), and callers without a
 * dsg_ctx (dsg_create itself allocates).
 *
 * Given loads[n] and A[n] (device pointers, uint32, by vertex id) it orders
 * the vertices by (loads[v], v) and returns the first densest suffix of that
 * order: the suffix, taken among all n non-empty suffixes, whose edge count
 * (the sum of A over its vertices) divided by its vertex count is largest,
 * the largest such suffix on ties.  When A counts, for every vertex, its
 * neighbours later in that order, the edge count of a suffix is the number
 * of edges of the subgraph it induces.
 *   m: the sum of A[0..n-1] (the edges of the whole graph), below 2^48.  The
 *      result is undefined unless m equals that sum;
 *   result: device pointer to int64[5], written on `cuda_stream`:
 *     (edges, vertices) of the densest suffix (largest suffix on ties),
 *     the position of its first vertex in the order, that vertex's load,
 *     and a device status: 0, or DSG_ERR_TIMEOUT if a bounded wait gave up
 *     (then the first four values are undefined).
 * The call is asynchronous: it only enqueues kernels on `cuda_stream` and
 * never synchronises.  It returns DSG_ERR_INVALID when n < 1,
 * n > DSG_NOALLOC_MAX_VERTICES, m < 0, m >= 2^48 or a pointer is NULL, and
 * DSG_ERR_CUDA when a launch fails or when a CUDA error is already pending
 * on the calling thread (that error is left in place for its owner and
 * nothing is launched).  loads and A are read only.
 *
 * Scratch memory: one static device array of about 4.4 MB inside libdsg,
 * held by every GPU that loads the library until the process exits.  Every
 * call uses the same array and leaves its contents behind; each call clears
 * what must start from zero (its look-back words and control block) before
 * use, so results never depend on earlier calls.  Calls whose work overlaps
 * on the GPU (on different streams or from different host threads) race on
 * the array and must be ordered by the caller.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, once per device even when several host threads make that
 * first call together; make that first call before any stream capture. */
int dsg_densest_suffix_noalloc(const uint32_t *loads, const uint32_t *A, int64_t n, int64_t m,
                               int64_t *result, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DSG_H */
