// server.cu -- continuous-batching request loop over the refine step.
//
// A server owns `slots` workers; each worker is a host thread with its own
// CUDA stream and dsg_ctx.  Submitted requests (a graph plus T, variant and
// eps) are copied into the server and queued in arrival order.  A free
// worker admits the request at the head of the queue as soon as its device
// memory estimate fits what is left of the HBM budget, then uploads it, runs
// it and reads the results back on its own stream.  Requests that arrive
// while others are on the GPU are therefore admitted as slots and memory free
// up, and the work of different slots overlaps on the device.  Every request
// runs exactly the computation dsg_run performs on it alone.
//
// Compact requests (graphs that dsg_run would give to a single thread block)
// bypass the slots: one more worker gathers every compact request queued at
// the time it is free (up to kMaxBatch, within the budget) and runs them as
// one batch (dsg_upload_batch / dsg_run_batch, one launch per variant),
// then picks up the next ones -- continuous batching.  A batch that fails
// as a whole (a malformed graph, a load overflow) is rerun one request at a
// time, so a bad request fails alone.
//
// PaRGreedy++ on a large graph is one cooperative launch whose blocks meet
// at grid-wide barriers, so all its blocks must be resident at once.  Each
// slot caps that grid at (SM count / slots) SMs' worth of blocks, so the
// grids of all slots fit the GPU together and their barriers never wait on
// one another's residency.
// The rounds are latency-bound, so the cap costs little per request and the
// slots' peels overlap.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <algorithm>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dsg.h"
#include "internal.h"
#include "peeling.h"

namespace {

using clock_type = std::chrono::steady_clock;

double ms_between(clock_type::time_point a, clock_type::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t id = 0;
    int64_t n = 0, m = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> adj;
    int variant = DSG_SORTING;
    int32_t T = 1;
    int64_t p = 0, q = 1;
    int64_t bytes = 0;
    clock_type::time_point t_submit, t_start, t_end;
    bool done = false;
    int status = DSG_OK;
    int slot = -1;
    dsg_result res{};
    std::vector<int64_t> loads;
    std::vector<int32_t> set;
    std::string err;
};

// device memory a request may hold at its peak: the CSR and its oriented
// copy, the per-run buffers of either variant and upload temporaries
int64_t estimate_bytes(int64_t n, int64_t m)
{
    return 12 * (2 * m) + 128 * n + (4 << 20);
}

}  // namespace

struct dsg_server {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    uint64_t next_id = 1;
    bool stop = false;
    int64_t n_queued = 0, n_running = 0, n_done = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;     // requests for the slots
    std::deque<Request *> cqueue;    // compact requests for the batch worker
    int n_slots = 0;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<dsg_ctx *> ctxs;
};

namespace {

void run_request(dsg_ctx *ctx, Request *r)
{
    dsg_graph *g = nullptr;
    int rc = dsg_upload_csr(ctx, r->n, r->off.data(), r->adj.empty() ? nullptr : r->adj.data(), DSG_VALIDATE, &g);
    if (rc == DSG_OK) {
        r->loads.assign((size_t)r->n, 0);
        r->set.assign((size_t)r->n, 0);
        r->res.flags = 0;
        r->res.loads = r->loads.data();
        r->res.best_set = r->set.data();
        r->res.trace = nullptr;
        rc = dsg_run(g, r->variant, r->T, r->p, r->q, nullptr, &r->res);
        dsg_free_graph(g);
    }
    r->status = rc;
    if (rc != DSG_OK) r->err = dsg_last_error(ctx);
    else r->set.resize((size_t)r->res.best_set_size);
}

constexpr size_t kMaxBatch = 1024;

// one batched run of compact requests of one variant; false if the batch
// failed as a whole
bool run_batch_group(dsg_ctx *ctx, int variant, const std::vector<Request *> &grp)
{
    const int32_t G = (int32_t)grp.size();
    std::vector<int64_t> n_per(G), p(G), q(G);
    std::vector<const int64_t *> offs(G);
    std::vector<const int32_t *> adjs(G);
    std::vector<int32_t> T(G);
    static const int32_t no_arcs = 0;
    int64_t N = 0;
    for (int32_t g = 0; g < G; ++g) {
        Request *r = grp[g];
        n_per[g] = r->n;
        offs[g] = r->off.data();
        adjs[g] = r->adj.empty() ? &no_arcs : r->adj.data();
        T[g] = r->T;
        p[g] = r->p;
        q[g] = r->q;
        N += r->n;
    }
    dsg_batch *b = nullptr;
    if (dsg_upload_batch(ctx, G, n_per.data(), offs.data(), adjs.data(), DSG_VALIDATE, &b) != DSG_OK) return false;
    std::vector<int64_t> best(4 * (size_t)G), loads((size_t)N);
    std::vector<int32_t> sets((size_t)N);
    dsg_batch_result out{};
    out.flags = 0;
    out.best = best.data();
    out.loads = loads.data();
    out.sets = sets.data();
    const int rc = dsg_run_batch(b, variant, T.data(), p.data(), q.data(), 0, &out);
    dsg_free_batch(b);
    if (rc != DSG_OK) return false;
    int64_t vb = 0;
    for (int32_t g = 0; g < G; ++g) {
        Request *r = grp[g];
        r->res.best_edges = best[4 * g];
        r->res.best_vertices = best[4 * g + 1];
        r->res.best_iter = (int32_t)best[4 * g + 2];
        r->res.best_set_size = best[4 * g + 3];
        r->loads.assign(loads.begin() + vb, loads.begin() + vb + r->n);
        r->set.assign(sets.begin() + vb, sets.begin() + vb + r->res.best_set_size);
        r->status = DSG_OK;
        vb += r->n;
    }
    return true;
}

void finish_requests(dsg_server *s, const std::vector<Request *> &rs)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request *r : rs) {
            r->t_end = clock_type::now();
            r->done = true;
            std::vector<int64_t>().swap(r->off);
            std::vector<int32_t>().swap(r->adj);
            s->in_use -= r->bytes;
            --s->n_running;
            ++s->n_done;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void batch_loop(dsg_server *s)
{
    cudaSetDevice(s->device);
    dsg_ctx *ctx = s->ctxs[s->n_slots];
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->cqueue.empty() && s->in_use + s->cqueue.front()->bytes <= s->budget);
            });
            if (s->stop) return;
            while (!s->cqueue.empty() && batch.size() < kMaxBatch &&
                   s->in_use + s->cqueue.front()->bytes <= s->budget) {
                Request *r = s->cqueue.front();
                s->cqueue.pop_front();
                s->in_use += r->bytes;
                --s->n_queued;
                ++s->n_running;
                r->t_start = clock_type::now();
                r->slot = s->n_slots;
                batch.push_back(r);
            }
        }
        for (int variant : {DSG_SORTING, DSG_PEELING}) {
            std::vector<Request *> grp;
            for (Request *r : batch)
                if (r->variant == variant) grp.push_back(r);
            if (grp.empty()) continue;
            if (!run_batch_group(ctx, variant, grp))
                for (Request *r : grp) run_request(ctx, r);
        }
        finish_requests(s, batch);
    }
}

void worker_loop(dsg_server *s, int slot)
{
    cudaSetDevice(s->device);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->queue.empty() &&
                                   s->in_use + s->queue.front()->bytes <= s->budget);
            });
            if (s->stop) return;
            r = s->queue.front();
            s->queue.pop_front();
            s->in_use += r->bytes;
            --s->n_queued;
            ++s->n_running;
            r->t_start = clock_type::now();
            r->slot = slot;
        }
        run_request(s->ctxs[slot], r);
        finish_requests(s, {r});
    }
}

}  // namespace

extern "C" {

int dsg_server_create(int device, int32_t slots, int64_t hbm_budget_bytes, dsg_server **out)
{
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes < 0) return DSG_ERR_INVALID;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return DSG_ERR_CUDA;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return DSG_ERR_CUDA;
    dsg_server *s = new (std::nothrow) dsg_server;
    if (!s) return DSG_ERR_NOMEM;
    s->device = device;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (int64_t)(free_b / 2);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
        delete s;
        return DSG_ERR_CUDA;
    }
    s->n_slots = slots;
    for (int i = 0; i <= slots; ++i) {       // slots, then the batch worker
        cudaStream_t st;
        dsg_ctx *c = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            dsg_server_destroy(s);
            return DSG_ERR_CUDA;
        }
        int rc = dsg_create(device, st, &c);
        if (rc != DSG_OK) {
            cudaStreamDestroy(st);
            dsg_server_destroy(s);
            return rc;
        }
        dsg::ctx_set_peel_max_blocks(c, std::max(1, sms / slots));
        s->streams.push_back(st);
        s->ctxs.push_back(c);
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_loop, s, i);
    s->workers.emplace_back(batch_loop, s);
    *out = s;
    return DSG_OK;
}

int dsg_server_submit(dsg_server *s, int64_t n, const int64_t *offsets, const int32_t *adj,
                      int variant, int32_t T, int64_t eps_num, int64_t eps_den, uint64_t *ticket)
{
    if (!s || !offsets || !ticket || n < 1) return DSG_ERR_INVALID;
    if (variant != DSG_SORTING && variant != DSG_PEELING) return DSG_ERR_INVALID;
    if (T < 1 || eps_den < 1 || eps_num < 0) return DSG_ERR_INVALID;
    const int64_t arcs = offsets[n];
    if (arcs < 0 || (arcs & 1) || offsets[0] != 0 || (arcs > 0 && !adj)) return DSG_ERR_INVALID;
    Request *r = new (std::nothrow) Request;
    if (!r) return DSG_ERR_NOMEM;
    r->n = n;
    r->m = arcs / 2;
    r->off.assign(offsets, offsets + n + 1);
    if (arcs > 0) r->adj.assign(adj, adj + arcs);
    r->variant = variant;
    r->T = T;
    r->p = eps_num;
    r->q = eps_den;
    r->bytes = estimate_bytes(n, r->m);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->bytes > s->budget) {
            delete r;
            return DSG_ERR_NOMEM;
        }
        r->id = s->next_id++;
        r->t_submit = clock_type::now();
        s->reqs[r->id] = r;
        if (dsg::is_compact(r->n, arcs)) s->cqueue.push_back(r);
        else s->queue.push_back(r);
        ++s->n_queued;
        *ticket = r->id;
    }
    s->cv_work.notify_all();
    return DSG_OK;
}

int dsg_server_wait(dsg_server *s, uint64_t ticket, int64_t timeout_ms, dsg_server_result *out,
                    int64_t *loads, int32_t *best_set)
{
    if (!s || !out) return DSG_ERR_INVALID;
    Request *r = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->reqs.find(ticket) == s->reqs.end()) return DSG_ERR_INVALID;
        // looked up again at every wake-up: another thread waiting on the
        // same ticket may have released it in the meantime
        auto ready = [&] {
            auto f = s->reqs.find(ticket);
            return f == s->reqs.end() || f->second->done;
        };
        if (timeout_ms < 0) s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return DSG_ERR_BUSY;
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return DSG_ERR_INVALID;
        r = it->second;
        s->reqs.erase(it);
    }
    s->cv_done.notify_all();      // other waiters on this ticket see it released
    out->status = r->status;
    out->best_iter = r->res.best_iter;
    out->best_edges = r->res.best_edges;
    out->best_vertices = r->res.best_vertices;
    out->best_set_size = r->res.best_set_size;
    out->n = r->n;
    out->m = r->m;
    out->slot = r->slot;
    out->queue_ms = ms_between(r->t_submit, r->t_start);
    out->run_ms = ms_between(r->t_start, r->t_end);
    out->latency_ms = ms_between(r->t_submit, r->t_end);
    std::strncpy(out->error, r->err.c_str(), sizeof(out->error) - 1);
    out->error[sizeof(out->error) - 1] = 0;
    if (r->status == DSG_OK) {
        if (loads) std::memcpy(loads, r->loads.data(), sizeof(int64_t) * r->loads.size());
        if (best_set && !r->set.empty()) std::memcpy(best_set, r->set.data(), sizeof(int32_t) * r->set.size());
    }
    delete r;
    return DSG_OK;
}

int dsg_server_stats(dsg_server *s, int64_t *queued, int64_t *running, int64_t *done, int64_t *bytes_in_use,
                     int64_t *budget)
{
    if (!s) return DSG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = s->n_queued;
    if (running) *running = s->n_running;
    if (done) *done = s->n_done;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    if (budget) *budget = s->budget;
    return DSG_OK;
}

void dsg_server_destroy(dsg_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->reqs) delete kv.second;
    for (size_t i = 0; i < s->ctxs.size(); ++i) dsg_destroy(s->ctxs[i]);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
