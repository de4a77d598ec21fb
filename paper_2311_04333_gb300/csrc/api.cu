// api.cu -- the C ABI of libdsg (include/dsg.h): contexts, graph upload and
// the host orchestration of one run of T refine iterations.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <algorithm>
#include <numeric>

#include "batch.h"
#include "dsg.h"
#include "internal.h"
#include "peeling.h"
#include "prune.h"

using namespace dsg;

struct dsg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    bool profiling = false;
    double ms[DSG_PHASE_COUNT] = {0, 0, 0};
    int64_t launches[DSG_PHASE_COUNT] = {0, 0, 0};
    int64_t bytes[DSG_PHASE_COUNT] = {0, 0, 0};
    std::vector<cudaEvent_t> ev;     // event pool for profiling
    size_t ev_used = 0;
    struct Pending { size_t a, b; int phase; };
    std::vector<Pending> pending;
    int32_t *err_flags = nullptr;    // device scratch for validation
    unsigned long long *red = nullptr;  // device scratch for reductions
    int peel_max_blocks = 0;         // SMs the PaRGreedy++ grid may use (0: all of them)
    int64_t peel_iters = 0, peel_rounds = 0, peel_work = 0;   // whole-GPU PaRGreedy++ telemetry
    cudaStream_t cap = nullptr;      // private stream that CUDA graphs are captured on
    // host uploads: the adjacency arrives in chunks on its own stream while
    // the context stream prepares the oriented copy; events [0, kUploadChunks)
    // mark the chunks, the last one the allocation they are copied into
    cudaStream_t copy = nullptr;
    cudaEvent_t up_ev[kUploadChunks + 1] = {};
    // test-only knobs of the bounded waits (dsg_debug_set)
    uint32_t dbg_spin_limit = 0;
    int32_t dbg_stall = 0;
};

namespace dsg {
void ctx_set_peel_max_blocks(dsg_ctx *ctx, int blocks) { ctx->peel_max_blocks = blocks; }
}  // namespace dsg

struct dsg_graph {
    dsg_ctx *ctx = nullptr;
    GraphDev g{};
    int64_t *off = nullptr;
    int32_t *adj = nullptr;
    WorkItem *items = nullptr;
    uint32_t *heavy_mem = nullptr;
    int64_t *ooff = nullptr;         // degree-oriented copy (sorting edge scan)
    uint32_t *oadj = nullptr;
    uint32_t *hub = nullptr;
    uint32_t *hot = nullptr;
    // run buffers, allocated on first use
    bool rb_ready = false;
    RunBufs rb{};
    void *rb_mem = nullptr;
    int64_t trace_cap = 0;
    int32_t *npass_log = nullptr;
    PeelBufs pb{};
    bool pb_ready = false;
    // whole-GPU structures (degree-oriented copy, chunk schedule): built at
    // upload for large graphs, on first use of the grid path for compact ones
    bool grid_ready = false;
    bool compact = false;
    int full_check = 0;
    // single-block path: parameters, run state and output staging
    void *bk_mem = nullptr;
    size_t bk_bytes = 0;
};

struct dsg_batch {
    dsg_ctx *ctx = nullptr;
    int32_t G = 0;
    int64_t N = 0, arcs = 0;
    std::vector<int64_t> maxdeg;     // per graph
    int64_t *vbase = nullptr, *off = nullptr;
    int32_t *adj = nullptr, *order = nullptr, *T = nullptr;
    int64_t *pq = nullptr;           // per graph eps = p / q
    uint32_t *graph_ctr = nullptr;
    void *run_mem = nullptr;         // loads, A, keys, ids, best_loads, staging
    size_t run_bytes = 0;
    int32_t thread_deg = 32;         // tuning (dsg_set_batch_tuning)
    int32_t block_deg = 1024;
};

namespace {

int fail(dsg_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(dsg_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? DSG_ERR_NOMEM : DSG_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);   \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// the device view of a pinned (page-locked, mapped) host pointer, or NULL
// for pageable memory
const void *pinned_view(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

// e1/v1 > e2/v2 (v > 0), exact
bool dens_gt_host(int64_t e1, int64_t v1, int64_t e2, int64_t v2)
{
    return (__int128)e1 * (__int128)v2 > (__int128)e2 * (__int128)v1;
}

cudaEvent_t ev_get(dsg_ctx *c)
{
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev.push_back(e);
    }
    return c->ev[c->ev_used++];
}

struct PhaseTimer {
    dsg_ctx *c;
    size_t a = 0;
    int phase;
    PhaseTimer(dsg_ctx *ctx, int ph) : c(ctx), phase(ph)
    {
        if (c->profiling) {
            a = c->ev_used;
            cudaEventRecord(ev_get(c), c->stream);
        }
    }
    ~PhaseTimer()
    {
        if (c->profiling) {
            size_t b = c->ev_used;
            cudaEventRecord(ev_get(c), c->stream);
            c->pending.push_back({a, b, phase});
        }
    }
};

void collect_timings(dsg_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev[p.a], c->ev[p.b]) == cudaSuccess) c->ms[p.phase] += ms;
    }
    c->pending.clear();
    c->ev_used = 0;
}

int ensure_run_bufs(dsg_ctx *ctx, dsg_graph *G, int32_t T)
{
    const int64_t n = G->g.n;
    RunBufs &b = G->rb;
    if (!G->rb_ready) {
        const int64_t ntiles = pass_tiles_last(n), stiles = pass_tiles_max(n);
        const int64_t nblk = (n + 4095) / 4096 + 1;
        size_t sz[12] = {
            (size_t)n * 4,                      // loads
            (size_t)n * 4,                      // A
            (size_t)n * 16,                     // keys[2], vals[2] (also output staging)
            (size_t)n * 4,                      // best_loads
            (size_t)stiles * kBuckets * 8,      // status
            (size_t)ntiles * kBuckets * 16,     // status_sum
            (size_t)ntiles * sizeof(Candidate), // cand
            sizeof(Control),                    // ctl
            (size_t)nblk * 8,                   // blk_a
            (size_t)nblk * 8,                   // blk_b
            (size_t)(G->g.n_hot > 0 ? G->g.n_hot : 1) * 8,  // hot_l, hot_c
            0};
        size_t total = 0;
        for (size_t s : sz) total += align256(s);
        char *mem = nullptr;
        CK(dev_malloc((void **)&mem, total, ctx->stream), "run buffers");
        char *p = mem;
        auto take = [&](size_t s) { char *q = p; p += align256(s); return (void *)q; };
        b.loads = (uint32_t *)take(sz[0]);
        b.A = (uint32_t *)take(sz[1]);
        uint32_t *kv = (uint32_t *)take(sz[2]);
        b.keys[0] = kv;
        b.keys[1] = kv + n;
        b.vals[0] = kv + 2 * n;
        b.vals[1] = kv + 3 * n;
        b.scratch = kv;
        b.best_loads = (uint32_t *)take(sz[3]);
        b.status = (unsigned long long *)take(sz[4]);
        b.status_sum = (unsigned long long *)take(sz[5]);
        b.cand = (Candidate *)take(sz[6]);
        b.ctl = (Control *)take(sz[7]);
        b.blk_a = (int64_t *)take(sz[8]);
        b.blk_b = (int64_t *)take(sz[9]);
        b.hot_l = (uint32_t *)take(sz[10]);
        b.hot_c = b.hot_l + (G->g.n_hot > 0 ? G->g.n_hot : 1);
        CK(cudaMemsetAsync(b.hot_c, 0, sizeof(uint32_t) * (size_t)(G->g.n_hot > 0 ? G->g.n_hot : 1), ctx->stream),
           "hot counters");
        b.ntiles = ntiles;
        b.nblk64 = nblk;
        // look-back words start at epoch 0, which no pass uses: memory that
        // held another graph's words (whose epochs restart with its own
        // control block) must not be taken for this graph's
        CK(cudaMemsetAsync(b.status, 0, sz[4], ctx->stream), "status init");
        CK(cudaMemsetAsync(b.status_sum, 0, sz[5], ctx->stream), "status sum init");
        CK(cudaMemsetAsync(b.ctl, 0, sizeof(Control), ctx->stream), "ctl init");
        CK(cudaMemsetAsync(b.A, 0, sz[1], ctx->stream), "A init");
        G->rb_mem = mem;
        G->rb_ready = true;
    }
    if (G->trace_cap < T) {
        if (b.trace) cudaFreeAsync(b.trace, ctx->stream);
        if (G->npass_log) cudaFreeAsync(G->npass_log, ctx->stream);
        b.trace = nullptr;
        G->npass_log = nullptr;
        CK(dev_malloc((void **)&b.trace, sizeof(int64_t) * 3 * (size_t)T, ctx->stream), "trace");
        CK(dev_malloc((void **)&G->npass_log, sizeof(int32_t) * (size_t)T, ctx->stream), "npass log");
        G->trace_cap = T;
    }
    return DSG_OK;
}

__global__ void k_log_npass(const Control *ctl, int32_t *log, int t) { log[t - 1] = ctl->npass; }

const char *const kGraphErr[5] = {"offsets are not non-decreasing", "a neighbour id is out of [0, n)",
                                  "the graph has a self-loop",
                                  "an adjacency list is not strictly ascending (duplicate or unsorted)",
                                  "the graph is not symmetric"};

// degree-oriented copy (with the adjacency checks fused into its count pass)
// and the chunk schedule of the vertices of large out-degree
int build_grid(dsg_ctx *ctx, dsg_graph *G, const UploadChunks *chunks)
{
    cudaError_t e;
    int32_t h_err[8];
    const int64_t n = G->g.n;
    int count_launches = 1;
    // on failure the oriented copy and the schedule are freed again, so that
    // a later call (the grid path of a compact graph is built on its first
    // grid run) starts from nothing
    auto undo = [&](int code) {
        cudaStream_t s = ctx->stream;
        if (G->ooff) cudaFreeAsync(G->ooff, s);
        if (G->oadj) cudaFreeAsync(G->oadj, s);
        if (G->hub) cudaFreeAsync(G->hub, s);
        if (G->hot) cudaFreeAsync(G->hot, s);
        if (G->items) cudaFreeAsync(G->items, s);
        if (G->heavy_mem) cudaFreeAsync(G->heavy_mem, s);
        G->ooff = nullptr;
        G->oadj = nullptr;
        G->hub = G->hot = nullptr;
        G->items = nullptr;
        G->heavy_mem = nullptr;
        G->g.ooff = nullptr;
        G->g.oadj = nullptr;
        G->g.hub_id = G->g.hot_id = nullptr;
        G->g.items = nullptr;
        G->g.heavy_acc = G->g.heavy_done = nullptr;
        return code;
    };
    // the count pass only raises flags: clear those another graph's upload
    // left (an upload's own offsets flag is already checked by now)
    if ((e = cudaMemsetAsync(ctx->err_flags, 0, 8 * sizeof(int32_t), ctx->stream)) != cudaSuccess)
        return undo(cuda_fail(ctx, e, "memset"));
    if ((e = build_orientation(G->g, ctx->stream, G->full_check, ctx->err_flags, &G->g.sorted, &G->ooff,
                               &G->oadj, &G->hub, &G->g.n_hub, &G->hot, &G->g.n_hot, chunks,
                               &count_launches)) != cudaSuccess)
        return undo(cuda_fail(ctx, e, "orientation"));
    cudaMemcpyAsync(h_err, ctx->err_flags, sizeof(h_err), cudaMemcpyDeviceToHost, ctx->stream);
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return undo(cuda_fail(ctx, e, "upload"));
    for (int i = 0; i < 5; ++i)
        if (h_err[i]) return undo(fail(ctx, DSG_ERR_INVALID, "invalid graph: %s", kGraphErr[i]));
    G->g.ooff = G->ooff;
    G->g.oadj = G->oadj;
    G->g.hub_id = G->hub;
    G->g.hot_id = G->hot;
    void *tmp = nullptr;
    const size_t tmp_bytes = (size_t)schedule_tmp_count(n) * sizeof(int64_t);
    if ((e = dev_malloc(&tmp, tmp_bytes, ctx->stream)) != cudaSuccess)
        return undo(cuda_fail(ctx, e, "schedule scratch"));
    GraphDev og = G->g;
    og.off = G->ooff;
    e = build_schedule(og, tmp, tmp_bytes, ctx->stream, &G->g.n_items, &G->g.n_heavy, &G->items, &G->heavy_mem);
    cudaFreeAsync(tmp, ctx->stream);
    if (e != cudaSuccess) return undo(cuda_fail(ctx, e, "schedule"));
    G->g.items = G->items;
    G->g.heavy_acc = G->heavy_mem;
    G->g.heavy_done = G->heavy_mem + (G->g.n_heavy > 0 ? G->g.n_heavy : 1);
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return undo(cuda_fail(ctx, e, "upload"));
    ctx->launches[DSG_PHASE_OTHER] += 4 + count_launches;
    G->grid_ready = true;
    return DSG_OK;
}

// parameters of a one-graph launch of the batch kernel
struct BlockParams {
    int64_t vbase[2];
    int64_t pq[2];
    int32_t T, order;
    uint32_t ctr, pad;
};

// All T iterations in one thread block (the batched form's kernel on one
// graph): no grid-wide synchronisation and a single launch per run.
int run_block(dsg_ctx *ctx, dsg_graph *G, int variant, int32_t T, int64_t p, int64_t q,
              const int64_t *init_loads, bool init_dev, dsg_result *out)
{
    const int64_t n = G->g.n;
    cudaStream_t s = ctx->stream;
    const bool dst_dev = out->flags & DSG_DST_DEVICE;
    const size_t need = align256(sizeof(BlockParams)) + 4 * align256(4 * (size_t)n) + 2 * align256(8 * (size_t)n)
                      + 2 * align256(8 * (size_t)n) + align256(4 * (size_t)n) + align256(32)
                      + align256(24 * (size_t)T);
    if (G->bk_bytes < need) {
        if (G->bk_mem) cudaFreeAsync(G->bk_mem, s);
        G->bk_mem = nullptr;
        G->bk_bytes = 0;
        CK(dev_malloc(&G->bk_mem, need, s), "block-path buffers");
        G->bk_bytes = need;
    }
    char *mp = (char *)G->bk_mem;
    auto take = [&](size_t b) { char *r = mp; mp += align256(b); return (void *)r; };
    BlockParams *prm = (BlockParams *)take(sizeof(BlockParams));
    BatchDev bd{};
    bd.G = 1;
    bd.Tmax = T;
    bd.vbase = prm->vbase;
    bd.off = G->off;
    bd.adj = G->adj;
    bd.order = &prm->order;
    bd.T = &prm->T;
    bd.pq = prm->pq;
    bd.loads = (uint32_t *)take(4 * (size_t)n);
    bd.A = (uint32_t *)take(4 * (size_t)n);
    bd.best_loads = (uint32_t *)take(4 * (size_t)n);
    bd.round = (uint32_t *)take(4 * (size_t)n);
    bd.keys = (uint32_t *)take(8 * (size_t)n);
    bd.ids = (uint32_t *)take(8 * (size_t)n);
    int64_t *st_init = (int64_t *)take(8 * (size_t)n);
    int64_t *st_loads = (int64_t *)take(8 * (size_t)n);
    int32_t *st_set = (int32_t *)take(4 * (size_t)n);
    int64_t *st_best = (int64_t *)take(32);
    int64_t *st_trace = (int64_t *)take(24 * (size_t)T);
    bd.init = nullptr;
    if (init_loads) {
        if (init_dev) bd.init = init_loads;
        else {
            CK(cudaMemcpyAsync(st_init, init_loads, 8 * (size_t)n, cudaMemcpyHostToDevice, s), "init loads copy");
            bd.init = st_init;
        }
    }
    bd.loads_out = out->loads ? (dst_dev ? out->loads : st_loads) : nullptr;
    bd.sets = out->best_set ? (dst_dev ? out->best_set : st_set) : nullptr;
    bd.best = st_best;
    bd.trace = out->trace ? (dst_dev ? out->trace : st_trace) : nullptr;
    BlockParams h{};
    h.vbase[0] = 0;
    h.vbase[1] = n;
    h.pq[0] = p;
    h.pq[1] = q;
    h.T = T;
    h.order = 0;
    CK(cudaMemcpyAsync(prm, &h, sizeof h, cudaMemcpyHostToDevice, s), "parameters");
    const int threads = n <= 1024 ? 256 : (n <= 8192 ? 512 : 1024);
    {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        CK(launch_batch(bd, variant, threads, ctx->sm_count, &prm->ctr, s), "block-path kernel");
    }
    ctx->launches[DSG_PHASE_OTHER] += 2;
    int64_t best[4];
    CK(cudaMemcpyAsync(best, st_best, 32, cudaMemcpyDeviceToHost, s), "best D2H");
    if (!dst_dev) {
        if (out->loads) CK(cudaMemcpyAsync(out->loads, st_loads, 8 * (size_t)n, cudaMemcpyDeviceToHost, s), "loads D2H");
        if (out->trace) CK(cudaMemcpyAsync(out->trace, st_trace, 24 * (size_t)T, cudaMemcpyDeviceToHost, s), "trace D2H");
    }
    CK(cudaStreamSynchronize(s), "run");
    if (!dst_dev && out->best_set && best[3] > 0) {
        CK(cudaMemcpyAsync(out->best_set, st_set, 4 * (size_t)best[3], cudaMemcpyDeviceToHost, s), "set D2H");
        CK(cudaStreamSynchronize(s), "set D2H");
    }
    out->best_edges = best[0];
    out->best_vertices = best[1];
    out->best_iter = (int32_t)best[2];
    out->best_set_size = best[3];
    if (ctx->profiling) collect_timings(ctx);
    return DSG_OK;
}

}  // namespace

extern "C" {

int dsg_create(int device, void *cuda_stream, dsg_ctx **out)
{
    if (!out) return DSG_ERR_INVALID;
    *out = nullptr;
    // the host-side context first: its failure touches no device
    dsg_ctx *ctx = host_alloc_fault() ? nullptr : new (std::nothrow) dsg_ctx;
    if (!ctx) return DSG_ERR_NOMEM;
    auto bail = [&](int code) { delete ctx; return code; };
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bail(DSG_ERR_CUDA);
    if (device < 0 || device >= ndev) return bail(DSG_ERR_INVALID);
    if (cudaSetDevice(device) != cudaSuccess) return bail(DSG_ERR_CUDA);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return bail(DSG_ERR_CUDA);
    if (prop.major * 10 + prop.minor < 100) return bail(DSG_ERR_INVALID);   // built for sm_103a only
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->sm_count = prop.multiProcessorCount;
    // Device memory is allocated stream-ordered from the device's default
    // pool.  Keep what is freed cached in the pool instead of returning it
    // to the driver at every synchronisation, so that uploading and freeing
    // graphs of tens of GB does not map and unmap physical memory each time
    // (dsg_destroy trims the pool).
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (host_alloc_fault() || cudaMalloc((void **)&ctx->err_flags, 64) != cudaSuccess ||
        cudaMalloc((void **)&ctx->red, 64) != cudaSuccess) {
        if (ctx->err_flags) cudaFree(ctx->err_flags);
        return bail(DSG_ERR_NOMEM);
    }
    *out = ctx;
    return DSG_OK;
}

void dsg_destroy(dsg_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    cudaFree(ctx->err_flags);
    cudaFree(ctx->red);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->copy) {
        cudaStreamSynchronize(ctx->copy);
        cudaStreamDestroy(ctx->copy);
        for (auto e : ctx->up_ev) if (e) cudaEventDestroy(e);
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    delete ctx;
}

const char *dsg_last_error(const dsg_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int dsg_debug_set(dsg_ctx *ctx, int knob, int64_t value)
{
    switch (knob) {
    case DSG_DEBUG_SPIN_LIMIT:
        if (!ctx || value < 0 || value > 0xffffffffll) return DSG_ERR_INVALID;
        ctx->dbg_spin_limit = (uint32_t)value;
        return DSG_OK;
    case DSG_DEBUG_STALL:
        if (!ctx || value < 0 || value > 2) return DSG_ERR_INVALID;
        ctx->dbg_stall = (int32_t)value;
        return DSG_OK;
    case DSG_DEBUG_FAIL_ALLOC:
        if (value < 0) return DSG_ERR_INVALID;
        set_alloc_fault(value);
        return DSG_OK;
    case DSG_DEBUG_FAIL_UPLOAD:
        if (value < 0) return DSG_ERR_INVALID;
        set_upload_fault(value);
        return DSG_OK;
    case DSG_DEBUG_PEEL_BLOCKS:
        if (!ctx || value < 0 || value > 65535) return DSG_ERR_INVALID;
        ctx->peel_max_blocks = (int)value;
        return DSG_OK;
    default:
        return ctx ? fail(ctx, DSG_ERR_INVALID, "unknown debug knob %d", knob) : DSG_ERR_INVALID;
    }
}

int dsg_upload_csr(dsg_ctx *ctx, int64_t n, const int64_t *offsets, const int32_t *adj,
                   uint32_t flags, dsg_graph **out)
{
    if (!ctx || !out) return DSG_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, DSG_ERR_INVALID, "n = %lld out of [1, 2^31)", (long long)n);
    if (!offsets) return fail(ctx, DSG_ERR_INVALID, "offsets is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const bool dev_src = flags & DSG_SRC_DEVICE;
    int64_t ends[2];
    if (dev_src) {
        CK(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, ctx->stream), "read offsets");
        CK(cudaMemcpyAsync(&ends[1], offsets + n, 8, cudaMemcpyDeviceToHost, ctx->stream), "read offsets");
        CK(cudaStreamSynchronize(ctx->stream), "sync");
    } else {
        ends[0] = offsets[0];
        ends[1] = offsets[n];
    }
    if (ends[0] != 0) return fail(ctx, DSG_ERR_INVALID, "offsets[0] = %lld, expected 0", (long long)ends[0]);
    const int64_t arcs = ends[1];
    if (arcs < 0 || (arcs & 1) || arcs >= ((int64_t)1 << 40))
        return fail(ctx, DSG_ERR_INVALID, "offsets[n] = %lld must be even and in [0, 2^40)", (long long)arcs);
    if (arcs > 0 && !adj) return fail(ctx, DSG_ERR_INVALID, "adj is NULL");

    // a large host graph is copied in vertex-range chunks on the context's
    // copy stream, overlapped with the preparation of the oriented copy
    const bool chunked = !dev_src && !is_compact(n, arcs) && arcs >= kChunkedUploadArcs;
    bool chunks_issued = false;
    UploadChunks chunks;
    dsg_graph *G = new (std::nothrow) dsg_graph;
    if (!G) return fail(ctx, DSG_ERR_NOMEM, "host allocation");
    G->ctx = ctx;
    auto bail = [&](int code) {
        // chunks still in flight finish before their buffer is freed
        if (chunks_issued) cudaStreamWaitEvent(ctx->stream, ctx->up_ev[kUploadChunks - 1], 0);
        if (G->off) cudaFreeAsync(G->off, ctx->stream);
        if (G->adj) cudaFreeAsync(G->adj, ctx->stream);
        if (G->items) cudaFreeAsync(G->items, ctx->stream);
        if (G->heavy_mem) cudaFreeAsync(G->heavy_mem, ctx->stream);
        if (G->ooff) cudaFreeAsync(G->ooff, ctx->stream);
        if (G->oadj) cudaFreeAsync(G->oadj, ctx->stream);
        if (G->hub) cudaFreeAsync(G->hub, ctx->stream);
        if (G->hot) cudaFreeAsync(G->hot, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        delete G;
        return code;
    };
    cudaError_t e;
    const cudaMemcpyKind kind = dev_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if ((e = dev_malloc((void **)&G->off, sizeof(int64_t) * (size_t)(n + 1), ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "offsets allocation"));
    if ((e = dev_malloc((void **)&G->adj, sizeof(int32_t) * (size_t)(arcs > 0 ? arcs : 1), ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "adjacency allocation"));
    if (!dev_src && upload_fault()) return bail(fail(ctx, DSG_ERR_CUDA, "offsets copy: injected upload failure"));
    // pinned host arrays of a large graph are copied by the SMs (steady at the
    // link's rate, where the copy engines' rate varies several-fold)
    const void *off_view = (!dev_src && chunked) ? pinned_view(offsets) : nullptr;
    const void *adj_view = (!dev_src && chunked) ? pinned_view(adj) : nullptr;
    if (off_view) {
        if ((e = launch_copy_h2d(off_view, G->off, sizeof(int64_t) * (size_t)(n + 1), ctx->sm_count, ctx->stream)) !=
            cudaSuccess)
            return bail(cuda_fail(ctx, e, "offsets copy"));
    } else if ((e = cudaMemcpyAsync(G->off, offsets, sizeof(int64_t) * (size_t)(n + 1), kind, ctx->stream)) !=
               cudaSuccess) {
        return bail(cuda_fail(ctx, e, "offsets copy"));
    }
    if (!dev_src && arcs > 0 && upload_fault())
        return bail(fail(ctx, DSG_ERR_CUDA, "adjacency copy: injected upload failure"));
    if (chunked) {
        if (!ctx->copy) {
            if ((e = cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking)) != cudaSuccess)
                return bail(cuda_fail(ctx, e, "copy stream"));
            for (int i = 0; i <= kUploadChunks; ++i)
                if ((e = cudaEventCreateWithFlags(&ctx->up_ev[i], cudaEventDisableTiming)) != cudaSuccess)
                    return bail(cuda_fail(ctx, e, "upload events"));
        }
        // the copies start once the allocation is in place on the context stream
        if ((e = cudaEventRecord(ctx->up_ev[kUploadChunks], ctx->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->copy, ctx->up_ev[kUploadChunks], 0)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "upload ordering"));
        // chunk boundaries at vertices splitting the arcs evenly; the byte
        // ranges are clamped to [0, arcs) and non-decreasing whatever the
        // offsets hold (they are validated on the device before any use)
        chunks.k = kUploadChunks;
        chunks.v[0] = 0;
        chunks.v[kUploadChunks] = n;
        int64_t a[kUploadChunks + 1];
        a[0] = 0;
        a[kUploadChunks] = arcs;
        for (int i = 1; i < kUploadChunks; ++i) {
            const int64_t target = (int64_t)((__int128)arcs * i / kUploadChunks);
            int64_t lo = chunks.v[i - 1], hi = n;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (offsets[mid] < target) lo = mid + 1; else hi = mid;
            }
            chunks.v[i] = lo;
            a[i] = std::min(std::max(offsets[lo], a[i - 1]), arcs);
        }
        chunks_issued = true;   // from here on a failure waits for the last chunk event
        for (int i = 0; i < kUploadChunks; ++i) {
            const size_t cb = sizeof(int32_t) * (size_t)(a[i + 1] - a[i]);
            if ((a[i + 1] > a[i] &&
                 (e = adj_view ? launch_copy_h2d((const int32_t *)adj_view + a[i], G->adj + a[i], cb, ctx->sm_count,
                                                 ctx->copy)
                               : cudaMemcpyAsync(G->adj + a[i], adj + a[i], cb, cudaMemcpyHostToDevice, ctx->copy)) !=
                     cudaSuccess) ||
                (e = cudaEventRecord(ctx->up_ev[i], ctx->copy)) != cudaSuccess) {
                cudaEventRecord(ctx->up_ev[kUploadChunks - 1], ctx->copy);
                return bail(cuda_fail(ctx, e, "adjacency copy"));
            }
            chunks.ev[i] = ctx->up_ev[i];
        }
    } else if (arcs > 0 && (e = cudaMemcpyAsync(G->adj, adj, sizeof(int32_t) * (size_t)arcs, kind, ctx->stream)) != cudaSuccess) {
        return bail(cuda_fail(ctx, e, "adjacency copy"));
    }
    G->g.n = n;
    G->g.arcs = arcs;
    G->g.off = G->off;
    G->g.adj = G->adj;
    G->full_check = (flags & DSG_VALIDATE) ? 1 : 0;
    G->compact = is_compact(n, arcs);
    int32_t h_err[8];
    if (G->compact && !dev_src) {
        // offsets and degrees checked on the host; the adjacency by one kernel
        int64_t maxdeg = 0;
        for (int64_t u = 0; u < n; ++u) {
            const int64_t d = offsets[u + 1] - offsets[u];
            if (d < 0 || offsets[u + 1] > arcs) return bail(fail(ctx, DSG_ERR_INVALID, "invalid graph: %s", kGraphErr[0]));
            maxdeg = std::max(maxdeg, d);
        }
        G->g.max_degree = maxdeg;
        if ((e = cudaMemsetAsync(ctx->err_flags, 0, 8 * sizeof(int32_t), ctx->stream)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "memset"));
        if ((e = launch_validate_adjacency(G->g, G->full_check, ctx->err_flags, ctx->stream)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "validate"));
        cudaMemcpyAsync(h_err, ctx->err_flags, sizeof(h_err), cudaMemcpyDeviceToHost, ctx->stream);
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "upload"));
        for (int i = 1; i < 5; ++i)
            if (h_err[i]) return bail(fail(ctx, DSG_ERR_INVALID, "invalid graph: %s", kGraphErr[i]));
        G->g.sorted = h_err[5] ? 0 : 1;
        ctx->launches[DSG_PHASE_OTHER] += 2;
        *out = G;
        return DSG_OK;
    }
    // validation: offsets first (monotone, inside [0, 2m]); the adjacency
    // (ids in range, no self-loops; with DSG_VALIDATE also strictly ascending
    // lists and symmetry) is checked in the pass that orients the graph, or
    // on its own for a compact graph
    if ((e = launch_validate(G->g, G->full_check, ctx->err_flags, ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "validate"));
    if ((e = cudaMemsetAsync(ctx->red, 0, 8, ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));
    if ((e = launch_degree_max(G->off, n, ctx->red, ctx->stream)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "degree max"));
    unsigned long long h_maxdeg = 0;
    cudaMemcpyAsync(h_err, ctx->err_flags, sizeof(h_err), cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(&h_maxdeg, ctx->red, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "upload"));
    if (h_err[0]) return bail(fail(ctx, DSG_ERR_INVALID, "invalid graph: %s", kGraphErr[0]));
    G->g.max_degree = (int64_t)h_maxdeg;
    ctx->launches[DSG_PHASE_OTHER] += 2;
    if (G->compact) {
        if ((e = launch_validate_adjacency(G->g, G->full_check, ctx->err_flags, ctx->stream)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "validate"));
        cudaMemcpyAsync(h_err, ctx->err_flags, sizeof(h_err), cudaMemcpyDeviceToHost, ctx->stream);
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "upload"));
        for (int i = 1; i < 5; ++i)
            if (h_err[i]) return bail(fail(ctx, DSG_ERR_INVALID, "invalid graph: %s", kGraphErr[i]));
        G->g.sorted = h_err[5] ? 0 : 1;
        ctx->launches[DSG_PHASE_OTHER] += 1;
        *out = G;
        return DSG_OK;
    }
    const int rc = build_grid(ctx, G, chunked ? &chunks : nullptr);
    if (rc != DSG_OK) return bail(rc);
    *out = G;
    return DSG_OK;
}

int dsg_graph_info(const dsg_graph *G, int64_t *n, int64_t *m, int64_t *max_degree)
{
    if (!G) return DSG_ERR_INVALID;
    if (n) *n = G->g.n;
    if (m) *m = G->g.arcs / 2;
    if (max_degree) *max_degree = G->g.max_degree;
    return DSG_OK;
}

void dsg_free_graph(dsg_graph *G)
{
    if (!G) return;
    dsg_ctx *ctx = G->ctx;
    cudaSetDevice(ctx->device);
    cudaFreeAsync(G->off, ctx->stream);
    cudaFreeAsync(G->adj, ctx->stream);
    if (G->items) cudaFreeAsync(G->items, ctx->stream);
    if (G->heavy_mem) cudaFreeAsync(G->heavy_mem, ctx->stream);
    if (G->ooff) cudaFreeAsync(G->ooff, ctx->stream);
    if (G->oadj) cudaFreeAsync(G->oadj, ctx->stream);
    if (G->hub) cudaFreeAsync(G->hub, ctx->stream);
    if (G->hot) cudaFreeAsync(G->hot, ctx->stream);
    if (G->rb_mem) cudaFreeAsync(G->rb_mem, ctx->stream);
    if (G->rb.trace) cudaFreeAsync(G->rb.trace, ctx->stream);
    if (G->npass_log) cudaFreeAsync(G->npass_log, ctx->stream);
    if (G->bk_mem) cudaFreeAsync(G->bk_mem, ctx->stream);
    peel_free(G->pb, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    delete G;
}

int dsg_set_profiling(dsg_ctx *ctx, int on)
{
    if (!ctx) return DSG_ERR_INVALID;
    ctx->profiling = on != 0;
    return DSG_OK;
}

int dsg_get_peel_stats(dsg_ctx *ctx, int64_t *iterations, int64_t *rounds, int64_t *alive_sum, int reset)
{
    if (!ctx) return DSG_ERR_INVALID;
    if (iterations) *iterations = ctx->peel_iters;
    if (rounds) *rounds = ctx->peel_rounds;
    if (alive_sum) *alive_sum = ctx->peel_work;
    if (reset) ctx->peel_iters = ctx->peel_rounds = ctx->peel_work = 0;
    return DSG_OK;
}

int dsg_get_stats(dsg_ctx *ctx, double *ms, int64_t *launches, int64_t *bytes, int reset)
{
    if (!ctx) return DSG_ERR_INVALID;
    for (int i = 0; i < DSG_PHASE_COUNT; ++i) {
        if (ms) ms[i] = ctx->ms[i];
        if (launches) launches[i] = ctx->launches[i];
        if (bytes) bytes[i] = ctx->bytes[i];
    }
    if (reset)
        for (int i = 0; i < DSG_PHASE_COUNT; ++i) ctx->ms[i] = 0, ctx->launches[i] = 0, ctx->bytes[i] = 0;
    return DSG_OK;
}

int dsg_run(dsg_graph *G, int variant, int32_t T, int64_t eps_num, int64_t eps_den,
            const int64_t *init_loads, dsg_result *out)
{
    if (!G || !out) return DSG_ERR_INVALID;
    dsg_ctx *ctx = G->ctx;
    if (variant != DSG_SORTING && variant != DSG_PEELING)
        return fail(ctx, DSG_ERR_INVALID, "unknown variant %d", variant);
    if (T < 1) return fail(ctx, DSG_ERR_INVALID, "T = %d must be >= 1", T);
    if (eps_den < 1 || eps_num < 0) return fail(ctx, DSG_ERR_INVALID, "eps = %lld/%lld: need p >= 0, q >= 1",
                                                (long long)eps_num, (long long)eps_den);
    if (eps_num + eps_den >= ((int64_t)1 << 31))
        return fail(ctx, DSG_ERR_OVERFLOW, "p + q must be < 2^31");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int64_t n = G->g.n;
    const bool init_dev = out->flags & DSG_INIT_DEVICE;
    const bool dst_dev = out->flags & DSG_DST_DEVICE;
    // overflow check: loads stay below 2^32
    unsigned long long max_init = 0;
    if (init_loads) {
        if (init_dev) {
            int *neg = (int *)(ctx->red + 1);
            CK(cudaMemsetAsync(ctx->red, 0, 16, ctx->stream), "memset");
            CK(launch_max_u64_of_i64(init_loads, n, ctx->red, neg, ctx->stream), "init max");
            unsigned long long h[2];
            CK(cudaMemcpyAsync(h, ctx->red, 16, cudaMemcpyDeviceToHost, ctx->stream), "init max");
            CK(cudaStreamSynchronize(ctx->stream), "sync");
            if ((int)(h[1] & 0xffffffffu)) return fail(ctx, DSG_ERR_INVALID, "negative initial load");
            max_init = h[0];
            ctx->launches[DSG_PHASE_OTHER] += 1;
        } else {
            for (int64_t v = 0; v < n; ++v) {
                if (init_loads[v] < 0) return fail(ctx, DSG_ERR_INVALID, "negative initial load at %lld", (long long)v);
                if ((unsigned long long)init_loads[v] > max_init) max_init = init_loads[v];
            }
        }
    }
    if (max_init + (unsigned long long)T * (unsigned long long)G->g.max_degree >= (1ull << 32))
        return fail(ctx, DSG_ERR_OVERFLOW, "max(init) + T * max_degree = %llu does not fit 32-bit loads",
                    max_init + (unsigned long long)T * (unsigned long long)G->g.max_degree);
    if ((out->flags & DSG_PATH_GRID) && (out->flags & DSG_PATH_BLOCK))
        return fail(ctx, DSG_ERR_INVALID, "DSG_PATH_GRID and DSG_PATH_BLOCK are exclusive");
    const bool block_path = (out->flags & DSG_PATH_BLOCK) ||
                            (!(out->flags & DSG_PATH_GRID) && block_path_default(variant, n, G->g.arcs));
    if (block_path) return run_block(ctx, G, variant, T, eps_num, eps_den, init_loads, init_dev, out);
    if (!G->grid_ready) {
        const int rg = build_grid(ctx, G, nullptr);
        if (rg != DSG_OK) return rg;
    }
    int rc = ensure_run_bufs(ctx, G, T);
    if (rc) return rc;
    RunBufs &b = G->rb;
    cudaStream_t s = ctx->stream;
    const int64_t *init_ptr = nullptr;
    if (init_loads) {
        if (init_dev) init_ptr = init_loads;
        else {
            CK(cudaMemcpyAsync(b.scratch, init_loads, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, s),
               "init loads copy");
            init_ptr = (const int64_t *)b.scratch;
        }
    }
    const int64_t m = G->g.arcs / 2;
    b.spin_limit = ctx->dbg_spin_limit;
    b.debug_stall = ctx->dbg_stall;
    {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        CK(launch_init(G->g, b, init_ptr, 0, s), "init");
        ctx->launches[DSG_PHASE_OTHER] += 2;
    }
    if (variant == DSG_SORTING) {
        const int es_grid = ctx->sm_count * edge_scan_sm_count();   // also sets the kernel attributes
        radix_prepare();
        auto iterations = [&](cudaStream_t ss) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            for (int t = 1; t <= T && e == cudaSuccess; ++t) {
                {
                    PhaseTimer pt(ctx, DSG_PHASE_OTHER);
                    e = launch_plan(G->g, b, t, ss);
                    k_log_npass<<<1, 1, 0, ss>>>(b.ctl, G->npass_log, t);
                }
                if (e == cudaSuccess) {
                    PhaseTimer pt(ctx, DSG_PHASE_EDGE_SCAN);
                    e = launch_edge_scan(G->g, b, es_grid, ss);
                }
                if (e == cudaSuccess) {
                    PhaseTimer pt(ctx, DSG_PHASE_SORT);
                    e = launch_asum_single_pass(G->g, b, ss);
                    if (e == cudaSuccess) e = launch_radix_passes(G->g, b, t, ss, nullptr, true, true);
                }
                if (e == cudaSuccess) {
                    PhaseTimer pt(ctx, DSG_PHASE_OTHER);
                    e = launch_snapshot(G->g, b, ss);
                }
                // the equal-loads edge scan is one of the two launches (one exits at
                // once); a hot tier adds its refresh and fold
                ctx->launches[DSG_PHASE_OTHER] += 3;
                ctx->launches[DSG_PHASE_EDGE_SCAN] += 2 + (G->g.n_hot > 0 ? 2 : 0);
                ctx->launches[DSG_PHASE_SORT] += kMaxPasses + 1;
                // oriented arcs (4m) + one target load per arc (4m) + oriented
                // offsets (8n) + own loads (4n) + A (4n)
                ctx->bytes[DSG_PHASE_EDGE_SCAN] += 8 * m + 16 * n;
            }
            return e;
        };
        // Below kGraphArcs the iteration's dozen launches cost more than
        // their work: the T iterations are captured once into a CUDA graph
        // (on a private stream, so any context stream works) and launched as
        // one on the context stream.
        if (!ctx->profiling && G->g.arcs <= kGraphArcs) {
            if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking), "capture stream");
            cudaGraph_t cg = nullptr;
            cudaGraphExec_t ge = nullptr;
            CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = iterations(ctx->cap);
            const cudaError_t ec = cudaStreamEndCapture(ctx->cap, &cg);
            if (e == cudaSuccess) e = ec;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, cg, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
            if (ge) cudaGraphExecDestroy(ge);     // freed once the launch completes
            if (cg) cudaGraphDestroy(cg);
            CK(e, "iterations (graph)");
        } else {
            CK(iterations(s), "iterations");
        }
    } else {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        int nl = 0;
        const int peel_blocks = ctx->peel_max_blocks > 0 ? ctx->peel_max_blocks : ctx->sm_count;
        rc = peel_run(ctx->stream, G->g, b, G->pb, G->pb_ready, ctx->sm_count, peel_blocks, T, eps_num, eps_den, &nl,
                      ctx->err);
        ctx->launches[DSG_PHASE_OTHER] += nl;
        if (rc) return rc;
    }
    // outputs: best set, loads, trace
    int nl = 0;
    // pinned host outputs are written by the kernels directly (no staging)
    int32_t *set_view = (!dst_dev && out->best_set) ? (int32_t *)pinned_view(out->best_set) : nullptr;
    int64_t *loads_view = (!dst_dev && out->loads) ? (int64_t *)pinned_view(out->loads) : nullptr;
    int32_t *set_dst = nullptr;
    if (out->best_set)
        set_dst = dst_dev ? out->best_set : (set_view ? set_view : (int32_t *)((char *)b.scratch + 8 * (size_t)n));
    {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        CK(launch_best_set(G->g, b, set_dst, s, &nl), "best set");
        if (out->loads) {
            int64_t *ldst = dst_dev ? out->loads : (loads_view ? loads_view : (int64_t *)b.scratch);
            CK(launch_loads_out(G->g, b, ldst, s), "loads out");
            ++nl;
            if (!dst_dev && !loads_view)
                CK(cudaMemcpyAsync(out->loads, ldst, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s), "loads D2H");
        }
        if (out->trace)
            CK(cudaMemcpyAsync(out->trace, b.trace, sizeof(int64_t) * 3 * (size_t)T,
                               dst_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "trace copy");
    }
    ctx->launches[DSG_PHASE_OTHER] += nl;
    Control h;
    CK(cudaMemcpyAsync(&h, b.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s), "control D2H");
    std::vector<int32_t> np(variant == DSG_SORTING ? T : 0);
    if (variant == DSG_SORTING)
        CK(cudaMemcpyAsync(np.data(), G->npass_log, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, s), "npass D2H");
    CK(cudaStreamSynchronize(s), "run");
    if (h.err) return fail(ctx, h.err, "device-side failure %d at site %d (a bounded wait gave up)", h.err, h.err_where);
    if (variant == DSG_PEELING) {
        ctx->peel_iters += T;
        ctx->peel_rounds += (int64_t)h.peel_rounds;
        ctx->peel_work += (int64_t)h.peel_work;
    }
    for (int32_t p : np) {
        // pass 0 reads (l, A) and writes l + A; scatter passes read and write
        // (key, value); the last pass reads only.
        int64_t by = 12 * n + (p > 1 ? 8 * n : 0) + (p > 2 ? 16 * n * (p - 2) : 0) + (p > 1 ? 8 * n : 0);
        ctx->bytes[DSG_PHASE_SORT] += by;
    }
    if (!dst_dev && out->best_set && h.set_size > 0 && !set_view) {
        CK(cudaMemcpyAsync(out->best_set, set_dst, sizeof(int32_t) * (size_t)h.set_size, cudaMemcpyDeviceToHost, s),
           "set D2H");
        CK(cudaStreamSynchronize(s), "set D2H");
    }
    out->best_edges = h.best_e;
    out->best_vertices = h.best_v;
    out->best_iter = h.best_iter;
    out->best_set_size = h.set_size;
    if (ctx->profiling) collect_timings(ctx);
    return DSG_OK;
}

int dsg_coreness(dsg_graph *G, int32_t *core, int64_t *k_max, uint32_t flags)
{
    if (!G || !core) return DSG_ERR_INVALID;
    dsg_ctx *ctx = G->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int64_t n = G->g.n;
    cudaStream_t s = ctx->stream;
    int rc = ensure_run_bufs(ctx, G, 1);
    if (rc) return rc;
    int32_t *dst = core;
    if (!(flags & DSG_DST_DEVICE)) CK(dev_malloc((void **)&dst, 4 * (size_t)n, s), "core buffer");
    int64_t km = 0;
    rc = coreness_run(s, G->g, G->rb.ctl, ctx->sm_count, dst, &km, ctx->err);
    if (rc == DSG_OK && !(flags & DSG_DST_DEVICE)) {
        cudaError_t e = cudaMemcpyAsync(core, dst, 4 * (size_t)n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "core copy");
    }
    if (!(flags & DSG_DST_DEVICE)) cudaFreeAsync(dst, s);
    if (rc == DSG_ERR_TIMEOUT) return fail(ctx, rc, "coreness: a bounded wait gave up");
    if (rc) return rc;
    if (k_max) *k_max = km;
    return DSG_OK;
}

// Alg. 1 with exact pruning (c_num == 0) or with pruning by the
// c-approximate decomposition (c = c_num / c_den): k-hat(v) is the smallest
// level tau_i >= core(v), so {v : k-hat(v) >= x} is the exact core of order
// apx_order(x) and every core this run takes is still a k-core by deletion.
// With exact_after (PaRApxGreedy++, Sec. 4: approximate pruning followed by
// exact pruning), the approximate levels only bracket k_max in
// (tau_{i-1}, tau_i]; k_max itself is then found exactly inside that bracket
// on the approximate core, and the run continues as with exact pruning.
static int run_pruned(dsg_graph *G, int variant, int32_t T, int64_t eps_num, int64_t eps_den, int64_t c_num,
                      int64_t c_den, dsg_result *out, dsg_prune_info *info, bool exact_after = false)
{
    if (!G || !out) return DSG_ERR_INVALID;
    dsg_ctx *ctx = G->ctx;
    bool apx = c_num != 0;
    if (apx && (c_den < 1 || c_num <= c_den || c_num >= ((int64_t)1 << 31)))
        return fail(ctx, DSG_ERR_INVALID, "c = %lld/%lld: need 1 <= c_den < c_num < 2^31", (long long)c_num,
                    (long long)c_den);
    if (variant != DSG_SORTING && variant != DSG_PEELING)
        return fail(ctx, DSG_ERR_INVALID, "unknown variant %d", variant);
    if (T < 1) return fail(ctx, DSG_ERR_INVALID, "T = %d must be >= 1", T);
    if (eps_den < 1 || eps_num < 0) return fail(ctx, DSG_ERR_INVALID, "eps = %lld/%lld: need p >= 0, q >= 1",
                                                (long long)eps_num, (long long)eps_den);
    if (eps_num + eps_den >= ((int64_t)1 << 31)) return fail(ctx, DSG_ERR_OVERFLOW, "p + q must be < 2^31");
    if (out->flags & (DSG_INIT_DEVICE | DSG_PATH_GRID | DSG_PATH_BLOCK))
        return fail(ctx, DSG_ERR_INVALID, "dsg_run_pruned starts from zero loads and picks the paths itself");
    if ((unsigned long long)T * (unsigned long long)G->g.max_degree >= (1ull << 32))
        return fail(ctx, DSG_ERR_OVERFLOW, "T * max_degree does not fit 32-bit loads");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int64_t n = G->g.n;
    cudaStream_t s = ctx->stream;
    const bool dst_dev = out->flags & DSG_DST_DEVICE;
    int rc = ensure_run_bufs(ctx, G, 1);
    if (rc) return rc;
    // buffers: core numbers, all loads (input ids), the best set (input ids),
    // the refine step's outputs (local ids)
    char *mem = nullptr;
    const size_t need = align256(4 * (size_t)n) + align256(8 * (size_t)n) + align256(4 * (size_t)n) +
                        align256(4 * (size_t)n) + align256(8 * (size_t)n) + align256(4 * (size_t)n);
    CK(dev_malloc((void **)&mem, need, s), "pruning buffers");
    int32_t *core = (int32_t *)mem;
    int64_t *loads_all = (int64_t *)(mem + align256(4 * (size_t)n));
    int32_t *sset = (int32_t *)((char *)loads_all + align256(8 * (size_t)n));
    int32_t *lset = (int32_t *)((char *)sset + align256(4 * (size_t)n));
    int64_t *nloads = (int64_t *)((char *)lset + align256(4 * (size_t)n));
    int32_t *kmask = (int32_t *)((char *)nloads + align256(8 * (size_t)n));
    CoreGraph cur;
    dsg_graph *cg = nullptr;
    std::vector<int64_t> trace(3 * (size_t)T, 0);
    auto finish = [&](int code) {
        if (cg) dsg_free_graph(cg);
        free_core(cur, s);
        cudaFreeAsync(mem, s);
        cudaStreamSynchronize(s);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(loads_all, 0, 8 * (size_t)n, s)) != cudaSuccess) return finish(cuda_fail(ctx, e, "memset"));
    // Alg. 1 set-up: k_max, L = ceil(k_max / 2), G <- L-core, S <- G.
    // Only cores of level >= ceil(k_max / 2) are ever used, and they lie in
    // H = G[deg >= k_low] for the bound k_low <= ceil(k_max / 2).  k_max is
    // the largest k whose k-core of H (by deletion) is not empty; each core
    // the loop needs is taken by deletion too, which is the set of vertices
    // whose core number in G reaches its level.
    int64_t kmax = 0, k_low = 0;
    KCoreBufs kb;
    int32_t *keep = kmask;
    // chain of nested cores (level, graph): chain[0] = G[deg >= k_low], each
    // next one the core of a higher level, taken from the one before
    std::vector<std::pair<int64_t, CoreGraph>> chain;
    auto kcore = [&](const CoreGraph &c, int64_t k, int64_t *alive) -> int {
        GraphDev cg_dev{};
        cg_dev.n = c.n;
        cg_dev.arcs = c.arcs;
        cg_dev.off = c.off;
        cg_dev.adj = c.adj;
        return kcore_run(s, cg_dev, G->rb.ctl, ctx->sm_count, kb, (int32_t)k, keep, alive, ctx->err);
    };
    auto done_k = [&](int code) {
        for (auto &c : chain) free_core(c.second, s);
        chain.clear();
        kcore_free(kb, s);
        return finish(code == DSG_ERR_TIMEOUT ? fail(ctx, code, "k-core: a bounded wait gave up") : code);
    };
    {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        CoreGraph H;
        if ((e = degree_core_bound(s, G->g, core, &k_low)) != cudaSuccess) return done_k(cuda_fail(ctx, e, "core bound"));
        if ((e = extract_core(s, n, G->g.off, G->g.adj, core, nullptr, k_low, nullptr, nullptr, &H)) != cudaSuccess)
            return done_k(cuda_fail(ctx, e, "degree core"));
        chain.push_back({k_low, H});
        // k_max: the largest k with a non-empty k-core; search upwards by
        // doubling from k_low, then by bisection.  The last core of the chain
        // is the lo-core, which holds every k-core with k >= lo, so each
        // success shrinks the graph later tests run on.  A k-core has k + 1
        // vertices and k (k + 1) / 2 edges: k_max < sqrt(2m) + 1.
        int64_t hi = (int64_t)std::sqrt(2.0 * (double)(G->g.arcs / 2)) + 2;
        hi = std::min(hi, G->g.max_degree + 1);
        int64_t lo = k_low;
        bool doubling = true;
        if (apx) hi = lo;      // the search below is the exact one
        while (hi - lo > 1) {
            const int64_t mid = doubling ? std::min(hi - 1, std::max<int64_t>(lo + 1, 2 * lo)) : lo + (hi - lo) / 2;
            int64_t alive = 0;
            const CoreGraph &C = chain.back().second;
            if ((rc = kcore(C, mid, &alive)) != DSG_OK) return done_k(rc);
            if (alive == 0) {
                hi = mid;
                doubling = false;
                continue;
            }
            lo = mid;
            CoreGraph nx;
            if ((e = extract_core(s, C.n, C.off, C.adj, keep, C.old_of, lo, nullptr, nullptr, &nx, true)) !=
                cudaSuccess)
                return done_k(cuda_fail(ctx, e, "core extraction"));
            chain.push_back({lo, nx});
        }
        kmax = lo;
        if (apx && G->g.arcs == 0) {
            kmax = 0;
        } else if (apx) {
            // k-hat_max, the smallest level >= k_max: probe the core orders
            // tau_i + 1 upwards from the first one >= k_low (the one below is
            // not empty: tau_{i-1} + 1 < k_low <= k_max); the first empty one
            // gives k_max <= tau_i
            int64_t tau = 1;
            while (tau + 1 < k_low) tau = apx_next_level(tau, c_num, c_den);
            for (;;) {
                int64_t alive = 0;
                const CoreGraph &C = chain.back().second;
                if ((rc = kcore(C, tau + 1, &alive)) != DSG_OK) return done_k(rc);
                if (alive == 0) break;
                CoreGraph nx;
                if ((e = extract_core(s, C.n, C.off, C.adj, keep, C.old_of, tau + 1, nullptr, nullptr, &nx, true)) !=
                    cudaSuccess)
                    return done_k(cuda_fail(ctx, e, "core extraction"));
                chain.push_back({tau + 1, nx});
                tau = apx_next_level(tau, c_num, c_den);
            }
            kmax = tau;
            if (exact_after) {
                // the exact stage: k_max in (level of the last core of the
                // chain, tau] by bisection over k-cores of that core
                int64_t lo2 = chain.back().first, hi2 = tau + 1;
                while (hi2 - lo2 > 1) {
                    const int64_t mid = lo2 + (hi2 - lo2) / 2;
                    int64_t alive = 0;
                    const CoreGraph &C = chain.back().second;
                    if ((rc = kcore(C, mid, &alive)) != DSG_OK) return done_k(rc);
                    if (alive == 0) {
                        hi2 = mid;
                        continue;
                    }
                    lo2 = mid;
                    CoreGraph nx;
                    if ((e = extract_core(s, C.n, C.off, C.adj, keep, C.old_of, lo2, nullptr, nullptr, &nx, true)) !=
                        cudaSuccess)
                        return done_k(cuda_fail(ctx, e, "core extraction"));
                    chain.push_back({lo2, nx});
                }
                kmax = lo2;
                apx = false;      // from here on: exact levels
            }
        }
    }
    // L = ceil(k_max / 2), or ceil(k-hat_max / (2c)) (the corollary on the
    // approximate k_max); G keeps the core of order `order`
    int64_t Ln = apx ? (kmax * c_den + 2 * c_num - 1) / (2 * c_num) : (kmax + 1) / 2, Ld = 1, level = Ln;
    int64_t order = apx ? apx_order(level, c_num, c_den) : level;
    {
        // the first core, from the highest core of the chain at or below its
        // order (the chain starts at G[deg >= k_low], which holds every core
        // of order >= k_low), or from G itself below k_low
        if (order >= chain[0].first) {
            size_t j = 0;
            for (size_t i = 0; i < chain.size(); ++i)
                if (chain[i].first <= order) j = i;
            const CoreGraph &C = chain[j].second;
            int64_t alive = 0;
            if ((rc = kcore(C, order, &alive)) != DSG_OK) return done_k(rc);
            if ((e = extract_core(s, C.n, C.off, C.adj, keep, C.old_of, order, nullptr, nullptr, &cur, true)) !=
                cudaSuccess)
                return done_k(cuda_fail(ctx, e, "core extraction"));
        } else {
            CoreGraph whole;
            whole.n = n;
            whole.arcs = G->g.arcs;
            whole.off = G->off;
            whole.adj = G->adj;
            int64_t alive = 0;
            if ((rc = kcore(whole, order, &alive)) != DSG_OK) return done_k(rc);
            if ((e = extract_core(s, n, G->off, G->adj, keep, nullptr, order, nullptr, nullptr, &cur, true)) !=
                cudaSuccess)
                return done_k(cuda_fail(ctx, e, "core extraction"));
        }
        for (auto &c : chain) free_core(c.second, s);
        chain.clear();
    }
    int64_t se = cur.arcs / 2, sv = cur.n, biter = 0, ssize = cur.n;
    if ((e = cudaMemcpyAsync(sset, cur.old_of, 4 * (size_t)cur.n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return done_k(cuda_fail(ctx, e, "set copy"));
    if (info) {
        info->k_max = kmax;
        info->core_vertices = cur.n;
        info->core_edges = cur.arcs / 2;
    }
    if ((rc = dsg_upload_csr(ctx, cur.n, cur.off, cur.adj, DSG_SRC_DEVICE, &cg)) != DSG_OK) return done_k(rc);
    for (int32_t t = 1; t <= T; ++t) {
        // Alg. 1 loop: one iteration of the refine step on the current core,
        // continuing its vertices' loads
        dsg_result r{};
        r.flags = DSG_DST_DEVICE | DSG_INIT_DEVICE;
        r.loads = nloads;
        r.best_set = lset;
        if ((rc = dsg_run(cg, variant, 1, eps_num, eps_den, cur.loads, &r)) != DSG_OK) return done_k(rc);
        if ((e = cudaMemcpyAsync(cur.loads, nloads, 8 * (size_t)cur.n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return done_k(cuda_fail(ctx, e, "loads copy"));
        trace[3 * (t - 1)] = r.best_edges;
        trace[3 * (t - 1) + 1] = r.best_vertices;
        trace[3 * (t - 1) + 2] = cur.n;
        // then keep a strictly denser result, raise L, re-prune
        if (!dens_gt_host(r.best_edges, r.best_vertices, se, sv)) continue;
        se = r.best_edges;
        sv = r.best_vertices;
        biter = t;
        ssize = r.best_set_size;
        if ((e = gather_ids(lset, ssize, cur.old_of, sset, s)) != cudaSuccess) return done_k(cuda_fail(ctx, e, "set"));
        if (dens_gt_host(se, sv, Ln, Ld)) {
            Ln = se;
            Ld = sv;
        }
        const int64_t nlevel = (Ln + Ld - 1) / Ld;
        if (nlevel <= level) continue;
        level = nlevel;
        const int64_t norder = apx ? apx_order(level, c_num, c_den) : level;
        if (norder <= order) continue;       // the same vertex set
        order = norder;
        CoreGraph nx;
        int64_t alive = 0;
        if ((rc = kcore(cur, order, &alive)) != DSG_OK) return done_k(rc);
        if ((e = extract_core(s, cur.n, cur.off, cur.adj, keep, cur.old_of, order, cur.loads, loads_all, &nx, true)) !=
            cudaSuccess)
            return done_k(cuda_fail(ctx, e, "core extraction"));
        free_core(cur, s);
        cur = nx;
        dsg_free_graph(cg);
        cg = nullptr;
        if ((rc = dsg_upload_csr(ctx, cur.n, cur.off, cur.adj, DSG_SRC_DEVICE, &cg)) != DSG_OK) return done_k(rc);
    }
    if ((e = scatter_loads(cur.loads, cur.n, cur.old_of, loads_all, s)) != cudaSuccess)
        return done_k(cuda_fail(ctx, e, "loads"));
    const cudaMemcpyKind k = dst_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (out->loads && (e = cudaMemcpyAsync(out->loads, loads_all, 8 * (size_t)n, k, s)) != cudaSuccess)
        return done_k(cuda_fail(ctx, e, "loads out"));
    if (out->best_set && ssize > 0 && (e = cudaMemcpyAsync(out->best_set, sset, 4 * (size_t)ssize, k, s)) != cudaSuccess)
        return done_k(cuda_fail(ctx, e, "set out"));
    if (out->trace &&
        (e = cudaMemcpyAsync(out->trace, trace.data(), 24 * (size_t)T,
                             dst_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s)) != cudaSuccess)
        return done_k(cuda_fail(ctx, e, "trace out"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done_k(cuda_fail(ctx, e, "pruned run"));
    out->best_edges = se;
    out->best_vertices = sv;
    out->best_iter = (int32_t)biter;
    out->best_set_size = ssize;
    if (info) {
        info->final_vertices = cur.n;
        info->L_num = Ln;
        info->L_den = Ld;
    }
    return done_k(DSG_OK);
}

int dsg_run_pruned(dsg_graph *G, int variant, int32_t T, int64_t eps_num, int64_t eps_den, dsg_result *out,
                   dsg_prune_info *info)
{
    return run_pruned(G, variant, T, eps_num, eps_den, 0, 1, out, info);
}

int dsg_run_pruned_apx(dsg_graph *G, int variant, int32_t T, int64_t eps_num, int64_t eps_den, int64_t c_num,
                       int64_t c_den, dsg_result *out, dsg_prune_info *info)
{
    if (G && c_num == 0) return fail(G->ctx, DSG_ERR_INVALID, "c_num = 0: use dsg_run_pruned");
    return run_pruned(G, variant, T, eps_num, eps_den, c_num, c_den, out, info);
}

int dsg_run_pruned_apx_exact(dsg_graph *G, int variant, int32_t T, int64_t eps_num, int64_t eps_den, int64_t c_num,
                             int64_t c_den, dsg_result *out, dsg_prune_info *info)
{
    if (G && c_num == 0) return fail(G->ctx, DSG_ERR_INVALID, "c_num = 0: use dsg_run_pruned");
    return run_pruned(G, variant, T, eps_num, eps_den, c_num, c_den, out, info, true);
}

int dsg_apx_coreness(dsg_graph *G, int64_t c_num, int64_t c_den, int32_t *core, int64_t *k_max, uint32_t flags)
{
    if (!G || !core) return DSG_ERR_INVALID;
    dsg_ctx *ctx = G->ctx;
    if (c_den < 1 || c_num <= c_den || c_num >= ((int64_t)1 << 31))
        return fail(ctx, DSG_ERR_INVALID, "c = %lld/%lld: need 1 <= c_den < c_num < 2^31", (long long)c_num,
                    (long long)c_den);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int64_t n = G->g.n;
    cudaStream_t s = ctx->stream;
    int rc = ensure_run_bufs(ctx, G, 1);
    if (rc) return rc;
    const bool dst_dev = flags & DSG_DST_DEVICE;
    char *mem = nullptr;
    CK(dev_malloc((void **)&mem, 3 * align256(4 * (size_t)n), s), "apx coreness buffers");
    int32_t *deg = (int32_t *)mem;
    int32_t *keep = (int32_t *)(mem + align256(4 * (size_t)n));
    int32_t *dst = dst_dev ? core : (int32_t *)(mem + 2 * align256(4 * (size_t)n));
    KCoreBufs kb;
    CoreGraph C;
    auto done = [&](int code) {
        free_core(C, s);
        kcore_free(kb, s);
        cudaFreeAsync(mem, s);
        cudaStreamSynchronize(s);
        return code == DSG_ERR_TIMEOUT ? fail(ctx, code, "approximate coreness: a bounded wait gave up") : code;
    };
    cudaError_t e;
    int64_t k_low = 0, khat = 0;
    // level by level: C is the (tau_{i-1} + 1)-core (the 1-core first: the
    // vertices with an edge); the vertices that its (tau_i + 1)-core drops
    // have core numbers in (tau_{i-1}, tau_i] and get tau_i
    if ((e = cudaMemsetAsync(dst, 0, 4 * (size_t)n, s)) != cudaSuccess) return done(cuda_fail(ctx, e, "memset"));
    if ((e = degree_core_bound(s, G->g, deg, &k_low)) != cudaSuccess) return done(cuda_fail(ctx, e, "degrees"));
    if ((e = extract_core(s, n, G->off, G->adj, deg, nullptr, 1, nullptr, nullptr, &C)) != cudaSuccess)
        return done(cuda_fail(ctx, e, "1-core"));
    int64_t tau = 1;
    while (C.n > 0) {
        GraphDev cd{};
        cd.n = C.n;
        cd.arcs = C.arcs;
        cd.off = C.off;
        cd.adj = C.adj;
        int64_t alive = 0;
        if ((rc = kcore_run(s, cd, G->rb.ctl, ctx->sm_count, kb, (int32_t)(tau + 1), keep, &alive, ctx->err)) !=
            DSG_OK)
            return done(rc);
        if (alive < C.n) khat = tau;
        if ((e = assign_removed(keep, C.n, C.old_of, (int32_t)tau, dst, s)) != cudaSuccess)
            return done(cuda_fail(ctx, e, "levels"));
        if (alive == 0) break;
        CoreGraph nx;
        if ((e = extract_core(s, C.n, C.off, C.adj, keep, C.old_of, tau + 1, nullptr, nullptr, &nx, true)) !=
            cudaSuccess)
            return done(cuda_fail(ctx, e, "core extraction"));
        free_core(C, s);
        C = nx;
        tau = apx_next_level(tau, c_num, c_den);
    }
    if (!dst_dev && (e = cudaMemcpyAsync(core, dst, 4 * (size_t)n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return done(cuda_fail(ctx, e, "core copy"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done(cuda_fail(ctx, e, "approximate coreness"));
    if (k_max) *k_max = khat;
    return done(DSG_OK);
}

int dsg_upload_batch(dsg_ctx *ctx, int32_t G, const int64_t *n_per, const int64_t *const *offsets,
                     const int32_t *const *adj, uint32_t flags, dsg_batch **out)
{
    if (!ctx || !out) return DSG_ERR_INVALID;
    *out = nullptr;
    if (G < 1 || !n_per || !offsets || !adj) return fail(ctx, DSG_ERR_INVALID, "G = %d: need G >= 1 and arrays", G);
    if (flags & DSG_SRC_DEVICE) return fail(ctx, DSG_ERR_INVALID, "dsg_upload_batch takes host arrays");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<int64_t> vbase(G + 1, 0), abase(G + 1, 0);
    std::vector<int64_t> maxdeg(G, 0);
    for (int32_t g = 0; g < G; ++g) {
        const int64_t n = n_per[g];
        if (n < 1) return fail(ctx, DSG_ERR_INVALID, "graph %d: n = %lld", g, (long long)n);
        if (!offsets[g] || offsets[g][0] != 0)
            return fail(ctx, DSG_ERR_INVALID, "graph %d: offsets must start at 0", g);
        const int64_t a = offsets[g][n];
        if (a < 0 || (a & 1)) return fail(ctx, DSG_ERR_INVALID, "graph %d: offsets[n] = %lld must be even", g, (long long)a);
        if (a > 0 && !adj[g]) return fail(ctx, DSG_ERR_INVALID, "graph %d: adj is NULL", g);
        for (int64_t v = 0; v < n; ++v) {
            const int64_t d = offsets[g][v + 1] - offsets[g][v];
            if (d < 0) return fail(ctx, DSG_ERR_INVALID, "graph %d: offsets are not non-decreasing", g);
            maxdeg[g] = std::max(maxdeg[g], d);
        }
        vbase[g + 1] = vbase[g] + n;
        abase[g + 1] = abase[g] + a;
    }
    const int64_t N = vbase[G], arcs = abase[G];
    if (N >= ((int64_t)1 << 31)) return fail(ctx, DSG_ERR_INVALID, "total vertices %lld >= 2^31", (long long)N);
    std::vector<int64_t> off(N + 1);
    std::vector<int32_t> adjp((size_t)std::max<int64_t>(arcs, 1));
    for (int32_t g = 0; g < G; ++g) {
        const int64_t n = n_per[g];
        for (int64_t v = 0; v < n; ++v) off[vbase[g] + v] = abase[g] + offsets[g][v];
        if (abase[g + 1] > abase[g])
            std::memcpy(adjp.data() + abase[g], adj[g], sizeof(int32_t) * (size_t)(abase[g + 1] - abase[g]));
    }
    off[N] = arcs;
    std::vector<int32_t> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (abase[a + 1] - abase[a]) + (vbase[a + 1] - vbase[a]) > (abase[b + 1] - abase[b]) + (vbase[b + 1] - vbase[b]);
    });
    dsg_batch *B = new (std::nothrow) dsg_batch;
    if (!B) return fail(ctx, DSG_ERR_NOMEM, "host allocation");
    B->ctx = ctx;
    B->G = G;
    B->N = N;
    B->arcs = arcs;
    B->maxdeg = maxdeg;
    auto bail = [&](int code) { dsg_free_batch(B); return code; };
    cudaError_t e;
    cudaStream_t st = ctx->stream;
    if ((e = dev_malloc((void **)&B->vbase, 8 * (size_t)(G + 1), st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->off, 8 * (size_t)(N + 1), st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->adj, 4 * adjp.size(), st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->order, 4 * (size_t)G, st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->T, 4 * (size_t)G, st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->pq, 16 * (size_t)G, st)) != cudaSuccess ||
        (e = dev_malloc((void **)&B->graph_ctr, 4, st)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "batch allocation"));
    if (upload_fault()) return bail(fail(ctx, DSG_ERR_CUDA, "batch copy: injected upload failure"));
    cudaMemcpyAsync(B->vbase, vbase.data(), 8 * (size_t)(G + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B->off, off.data(), 8 * (size_t)(N + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B->adj, adjp.data(), 4 * adjp.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B->order, order.data(), 4 * (size_t)G, cudaMemcpyHostToDevice, st);
    BatchDev bd{};
    bd.G = G;
    bd.vbase = B->vbase;
    bd.off = B->off;
    bd.adj = B->adj;
    if ((e = launch_batch_validate(bd, (flags & DSG_VALIDATE) ? 1 : 0, ctx->err_flags, st)) != cudaSuccess)
        return bail(cuda_fail(ctx, e, "batch validation"));
    int32_t h_err[8];
    cudaMemcpyAsync(h_err, ctx->err_flags, sizeof(h_err), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(ctx, e, "batch upload"));
    static const char *what[5] = {"offsets are not non-decreasing", "a neighbour id is out of [0, n)",
                                  "a graph has a self-loop",
                                  "an adjacency list is not strictly ascending (duplicate or unsorted)",
                                  "a graph is not symmetric"};
    for (int i = 0; i < 5; ++i)
        if (h_err[i]) return bail(fail(ctx, DSG_ERR_INVALID, "invalid batch: %s", what[i]));
    ctx->launches[DSG_PHASE_OTHER] += 1;
    *out = B;
    return DSG_OK;
}

int dsg_batch_info(const dsg_batch *b, int32_t *G, int64_t *total_n, int64_t *total_m)
{
    if (!b) return DSG_ERR_INVALID;
    if (G) *G = b->G;
    if (total_n) *total_n = b->N;
    if (total_m) *total_m = b->arcs / 2;
    return DSG_OK;
}

int dsg_run_batch(dsg_batch *Bt, int variant, const int32_t *T, const int64_t *eps_num,
                  const int64_t *eps_den, int32_t threads_per_graph, dsg_batch_result *out)
{
    if (!Bt || !out) return DSG_ERR_INVALID;
    dsg_ctx *ctx = Bt->ctx;
    if (variant != DSG_SORTING && variant != DSG_PEELING)
        return fail(ctx, DSG_ERR_INVALID, "variant %d: use DSG_SORTING or DSG_PEELING", variant);
    if (!T || !out->best) return fail(ctx, DSG_ERR_INVALID, "T and out->best are required");
    const int threads = threads_per_graph ? threads_per_graph : 512;
    if (threads != 256 && threads != 512 && threads != 1024)
        return fail(ctx, DSG_ERR_INVALID, "threads_per_graph = %d: use 256, 512 or 1024", threads_per_graph);
    int32_t Tmax = 0;
    std::vector<int64_t> pq(2 * (size_t)Bt->G);
    for (int32_t g = 0; g < Bt->G; ++g) {
        if (T[g] < 1) return fail(ctx, DSG_ERR_INVALID, "T[%d] = %d must be >= 1", g, T[g]);
        if ((unsigned long long)T[g] * (unsigned long long)Bt->maxdeg[g] >= (1ull << 32))
            return fail(ctx, DSG_ERR_OVERFLOW, "graph %d: T * max_degree does not fit 32-bit loads", g);
        Tmax = std::max(Tmax, T[g]);
        const int64_t p = eps_num ? eps_num[g] : 0, q = eps_den ? eps_den[g] : 1;
        if (variant == DSG_PEELING) {
            if (p < 0 || q < 1) return fail(ctx, DSG_ERR_INVALID, "graph %d: eps = %lld/%lld", g, (long long)p, (long long)q);
            if (p + q >= (1ll << 31)) return fail(ctx, DSG_ERR_OVERFLOW, "graph %d: p + q must stay below 2^31", g);
        }
        pq[2 * g] = p;
        pq[2 * g + 1] = q;
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = ctx->stream;
    const int64_t N = Bt->N, G = Bt->G;
    const bool dev = out->flags & DSG_DST_DEVICE;
    // run state (+ staging for host outputs)
    const size_t need = align256(4 * (size_t)N) * 4 + align256(8 * (size_t)N) * 2 + align256(8 * (size_t)N)
                      + align256(4 * (size_t)N) + align256(32 * (size_t)G) + align256(24 * (size_t)G * Tmax);
    if (Bt->run_bytes < need) {
        if (Bt->run_mem) cudaFreeAsync(Bt->run_mem, st);
        Bt->run_mem = nullptr;
        Bt->run_bytes = 0;
        CK(dev_malloc(&Bt->run_mem, need, st), "batch run buffers");
        Bt->run_bytes = need;
    }
    char *p = (char *)Bt->run_mem;
    auto take = [&](size_t b) { char *q = p; p += align256(b); return (void *)q; };
    BatchDev bd{};
    bd.G = (int32_t)G;
    bd.Tmax = Tmax;
    bd.vbase = Bt->vbase;
    bd.off = Bt->off;
    bd.adj = Bt->adj;
    bd.order = Bt->order;
    bd.T = Bt->T;
    bd.pq = Bt->pq;
    bd.init = nullptr;
    bd.loads = (uint32_t *)take(4 * (size_t)N);
    bd.A = (uint32_t *)take(4 * (size_t)N);
    bd.best_loads = (uint32_t *)take(4 * (size_t)N);
    bd.round = (uint32_t *)take(4 * (size_t)N);
    bd.keys = (uint32_t *)take(8 * (size_t)N);
    bd.ids = (uint32_t *)take(8 * (size_t)N);
    int64_t *st_loads = (int64_t *)take(8 * (size_t)N);
    int32_t *st_sets = (int32_t *)take(4 * (size_t)N);
    int64_t *st_best = (int64_t *)take(32 * (size_t)G);
    int64_t *st_trace = (int64_t *)take(24 * (size_t)G * Tmax);
    bd.loads_out = out->loads ? (dev ? out->loads : st_loads) : nullptr;
    bd.sets = out->sets ? (dev ? out->sets : st_sets) : nullptr;
    bd.best = dev ? out->best : st_best;
    bd.trace = out->trace ? (dev ? out->trace : st_trace) : nullptr;
    bd.thread_deg = Bt->thread_deg;
    bd.block_deg = Bt->block_deg;
    CK(cudaMemcpyAsync(Bt->T, T, 4 * (size_t)G, cudaMemcpyHostToDevice, st), "T copy");
    CK(cudaMemcpyAsync(Bt->pq, pq.data(), 16 * (size_t)G, cudaMemcpyHostToDevice, st), "eps copy");
    {
        PhaseTimer pt(ctx, DSG_PHASE_OTHER);
        CK(launch_batch(bd, variant, threads, ctx->sm_count, Bt->graph_ctr, st), "batch kernel");
    }
    ctx->launches[DSG_PHASE_OTHER] += 1;
    if (!dev) {
        CK(cudaMemcpyAsync(out->best, st_best, 32 * (size_t)G, cudaMemcpyDeviceToHost, st), "best D2H");
        if (out->loads) CK(cudaMemcpyAsync(out->loads, st_loads, 8 * (size_t)N, cudaMemcpyDeviceToHost, st), "loads D2H");
        if (out->sets) CK(cudaMemcpyAsync(out->sets, st_sets, 4 * (size_t)N, cudaMemcpyDeviceToHost, st), "sets D2H");
        if (out->trace) CK(cudaMemcpyAsync(out->trace, st_trace, 24 * (size_t)G * Tmax, cudaMemcpyDeviceToHost, st), "trace D2H");
    }
    CK(cudaStreamSynchronize(st), "batch run");
    if (ctx->profiling) collect_timings(ctx);
    return DSG_OK;
}

int dsg_set_batch_tuning(dsg_batch *b, int32_t thread_degree, int32_t block_degree)
{
    if (!b) return DSG_ERR_INVALID;
    if (thread_degree < 0 || thread_degree > (1 << 20) || block_degree < 0 || block_degree > (1 << 30))
        return fail(b->ctx, DSG_ERR_INVALID, "thread_degree = %d, block_degree = %d out of range", thread_degree,
                    block_degree);
    b->thread_deg = thread_degree ? thread_degree : 32;
    b->block_deg = block_degree ? block_degree : 1024;
    return DSG_OK;
}

void dsg_free_batch(dsg_batch *B)
{
    if (!B) return;
    dsg_ctx *ctx = B->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    if (B->vbase) cudaFreeAsync(B->vbase, st);
    if (B->off) cudaFreeAsync(B->off, st);
    if (B->adj) cudaFreeAsync(B->adj, st);
    if (B->order) cudaFreeAsync(B->order, st);
    if (B->T) cudaFreeAsync(B->T, st);
    if (B->pq) cudaFreeAsync(B->pq, st);
    if (B->graph_ctr) cudaFreeAsync(B->graph_ctr, st);
    if (B->run_mem) cudaFreeAsync(B->run_mem, st);
    cudaStreamSynchronize(st);
    delete B;
}

}  // extern "C"
