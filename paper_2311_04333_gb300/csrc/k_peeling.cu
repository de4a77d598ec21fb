// k_peeling.cu -- PaRGreedy++ refine step (arXiv 2311.04333, Sec. 3.3
// "ParallelGreedy++"): the ordering comes from bucketed peeling by the key
// l(v) + deg_H(v) with H reset to G each iteration.  Each round peels every
// alive vertex whose key is within a factor (1 + p/q) of the round's minimum
// key (key*q <= min*(p+q)), all at once; the degree decrements they cause are
// applied only after the round's set is fixed.  The order is (round, id).
//
// One cooperative persistent kernel runs all rounds of an iteration, two
// bounded grid barriers per round (three when F has vertices of degree
// above 512):
//   A:  every alive vertex publishes its key (kept as kv = l + deg_H and
//       decremented in place) in a snapshot word st = (round | key); grid
//       minimum of the keys;
//   BC: the round's set F = {key*q <= thr} is decided from the snapshots,
//       so a block can split its share of the alive list and at once process
//       the low-degree F vertices it found: for v in F, count its later
//       neighbours (alive ones not in F, and ones in F with a larger id)
//       -> A[v], l(v) += A[v], and decrement kv of the alive neighbours not
//       in F;
//   H:  the same for the heavier F vertices, whose arcs are cut into chunks
//       of 2,048 that all blocks share.
// Blocks of 512 threads, two per SM; they leave as the alive set shrinks
// (one block per 2,048 alive vertices or 32,768 of their arcs, whichever
// needs more), down to a single block
// that rounds with block barriers only.
// The densest suffix of the (round, id) order then reuses the radix passes
// of the sorting path with key = round and value = A (Alg. 3, suffix densities).
#include <mutex>

#include "common.cuh"
#include "dsg.h"
#include "peeling.h"

namespace dsg {

constexpr uint32_t kUnpeeled = 0xffffffffu;
constexpr int kPeelThreads = 512;
constexpr uint32_t kAlivePerBlock = 2048;   // blocks: one per this many alive vertices
constexpr int64_t kArcsPerBlock = 32768;    //   or per this many arcs of alive vertices
constexpr int64_t kLocalDegree = 512;       // F vertices up to this degree: the finding block
constexpr int64_t kPeelChunk = 2048;        // arcs per work item of the heavier F vertices
constexpr int kQueueCap = 4096;             // block-local queue of F vertices
constexpr int kSplitK = 2;                  // alive entries per thread per step of the split
// heavy-list words: (count or vertex) << 33 | chunk index; n < 2^31 and the
// chunks of one round are fewer than 2^40 / 2048 + n < 2^33
constexpr int kHeavyShift = 33;
constexpr unsigned long long kChunkMask = (1ull << kHeavyShift) - 1;

struct PeelCtl {
    unsigned long long mn[2];   // round minimum key, by round parity
    unsigned long long heavy[2];// heavy F vertices (bits 33..63) and their chunks (bits 0..32)
    uint32_t n_next[2];         // alive-list sizes, by round parity
    uint32_t rounds;
    uint32_t bar_count;         // barrier arrivals this iteration
    uint32_t abort;
    unsigned long long work;    // sum over rounds of the alive-list size
    unsigned long long arcs_alive;  // arcs of the alive vertices
};

// blocks worth keeping for na alive vertices holding `arcs` arcs
__host__ __device__ __forceinline__ uint32_t peel_blocks(uint64_t na, uint64_t arcs)
{
    const uint64_t a = (na + kAlivePerBlock - 1) / kAlivePerBlock, b = (arcs + kArcsPerBlock - 1) / kArcsPerBlock;
    const uint64_t x = a > b ? a : b;
    return x < 1 ? 1u : (x > 0xffffu ? 0xffffu : (uint32_t)x);
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Bounded barrier over the first `nb` blocks (co-resident: cooperative
// launch).  The arrival counter only grows during an iteration: every block
// adds nb to its own running target before each barrier, arrives, and waits
// until the counter reaches the target.  A single block needs only its own
// barrier.
__device__ __forceinline__ bool grid_barrier(PeelCtl *pc, Control *ctl, uint32_t nb, uint32_t &target)
{
    __shared__ int s_ok;
    __syncthreads();
    if (nb == 1) return true;
    target += nb;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        // (test-only: debug_stall 2 keeps block 1 from arriving at the first
        // barrier, so that every block's wait runs out)
        if (!(ctl->debug_stall == 2 && blockIdx.x == 1 && target == nb)) atomicAdd(&pc->bar_count, 1u);
        const uint32_t limit = spin_limit_of(ctl->spin_limit);
        uint32_t polls = 0;
        while (ld_acquire_u32(&pc->bar_count) < target) {
            if (++polls > limit || ((polls & 255) == 0 && ld_acquire_u32(&pc->abort))) {
                atomicExch(&pc->abort, 1u);
                set_error(ctl, DSG_ERR_TIMEOUT, 400);
                ok = 0;
                break;
            }
            if (polls > 64) __nanosleep(32);
        }
        if (ok && ld_acquire_u32(&pc->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void k_peel_init(const int64_t *__restrict__ off, const uint32_t *__restrict__ loads, int64_t n,
                            int64_t arcs, uint32_t *kv, uint32_t *round, uint32_t *list0, PeelCtl *pc)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        kv[v] = loads[v] + (uint32_t)(off[v + 1] - off[v]);
        round[v] = kUnpeeled;
        list0[v] = (uint32_t)v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pc->mn[0] = pc->mn[1] = ~0ull;
        pc->heavy[0] = pc->heavy[1] = 0;
        pc->n_next[0] = (uint32_t)n;
        pc->n_next[1] = 0;
        pc->rounds = 0;
        pc->bar_count = 0;
        pc->abort = 0;
        pc->work = 0;
        pc->arcs_alive = (unsigned long long)arcs;
    }
}

// warp-aggregated slot claim on a counter (all lanes call it)
__device__ __forceinline__ uint32_t warp_claim(bool pred, uint32_t *cnt)
{
    const uint32_t m = __ballot_sync(kFull, pred);
    if (!m) return 0;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    return base + __popc(m & lanemask_lt());
}

constexpr int64_t kTinyDegree = 8;          // F vertices up to this degree: thread per vertex

struct PeelSmem {
    unsigned long long red[kPeelThreads / 32];
    uint32_t queue[kQueueCap];              // F vertices of degree (kTinyDegree, kLocalDegree]
    uint32_t tiny[kQueueCap];               // F vertices of degree <= kTinyDegree
    uint32_t nq, nt;
    uint32_t nsurv, nbase;                  // survivors claimed by the block, their base in the next list
    unsigned long long arcs_gone;           // arcs of the block's F vertices this round
};

// later-neighbour count of one F vertex over arcs [s, e) with `stride`
// lanes starting at `first`; decrements kv of the alive neighbours not in F
__device__ __forceinline__ uint32_t count_arcs(const int32_t *__restrict__ adj, int64_t s, int64_t e, int first,
                                               int stride, uint32_t v, uint32_t r, unsigned long long thr,
                                               uint64_t q, const unsigned long long *st, uint32_t *kv)
{
    uint32_t c = 0;
    for (int64_t j = s + first; j < e; j += stride) {
        const uint32_t w = (uint32_t)adj[j];
        const unsigned long long sw = st[w];
        const uint32_t rw = (uint32_t)(sw >> 32);
        if (rw != kUnpeeled && rw != r) continue;             // peeled in an earlier round
        const bool w_in_f = rw == r || (sw & 0xffffffffull) * q <= thr;
        if (!w_in_f) {
            ++c;
            atomicSub(&kv[w], 1u);
        } else if (w > v) {
            ++c;
        }
    }
    return c;
}

// the block's queued F vertices of low degree: thread per vertex for the
// tiny ones, warp per vertex for the others
__device__ void drain_queue(PeelSmem &S, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            uint32_t r, unsigned long long thr, uint64_t q, const unsigned long long *st,
                            uint32_t *kv, uint32_t *loads, uint32_t *A)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kPeelThreads / 32;
    const uint32_t nt = S.nt;
    for (uint32_t f = threadIdx.x; f < nt; f += kPeelThreads) {
        const uint32_t v = S.tiny[f];
        const uint32_t c = count_arcs(adj, off[v], off[v + 1], 0, 1, v, r, thr, q, st, kv);
        A[v] = c;
        loads[v] += c;
    }
    const uint32_t nq = S.nq;
    for (uint32_t f = warp; f < nq; f += NW) {
        const uint32_t v = S.queue[f];
        uint32_t c = count_arcs(adj, off[v], off[v + 1], lane, 32, v, r, thr, q, st, kv);
        c = __reduce_add_sync(kFull, c);
        if (lane == 0) {
            A[v] = c;
            loads[v] += c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S.nq = 0;
        S.nt = 0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPeelThreads, 2)
k_peel(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int64_t n,
       uint32_t *loads, uint32_t *A, uint32_t *kv, unsigned long long *st, uint32_t *round,
       uint32_t *list0, uint32_t *list1, unsigned long long *heavy, uint64_t p, uint64_t q,
       PeelCtl *pc, Control *ctl, uint32_t *round_min, uint32_t fixed_k)
{
    __shared__ PeelSmem S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kPeelThreads / 32;
    uint32_t r = 0;
    uint32_t P = gridDim.x;                 // participating blocks
    uint32_t bar_target = 0;
    uint32_t na_prev = 0;
    if (tid == 0) {
        S.nq = 0;
        S.nt = 0;
        S.nsurv = 0;
        S.arcs_gone = 0;
    }
    for (;; ++r) {
        const uint32_t na = ld_acquire_u32(&pc->n_next[r & 1]);
        if (na == 0) break;
        // fixed threshold (k-core by deletion): stop once a round peels nothing
        if (fixed_k != kUnpeeled && r > 0 && na == na_prev) break;
        na_prev = na;
        P = min(P, peel_blocks(na, ld_acquire_u64(&pc->arcs_alive)));
        if (blockIdx.x >= P) break;
        uint32_t *cur = (r & 1) ? list1 : list0;
        uint32_t *nxt = (r & 1) ? list0 : list1;
        if (blockIdx.x == 0 && tid == 0) {
            pc->n_next[(r + 1) & 1] = 0;
            pc->mn[(r + 1) & 1] = ~0ull;
            pc->heavy[(r + 1) & 1] = 0;
            pc->work += na;
        }
        const uint32_t stride = P * kPeelThreads;
        // ---- A: snapshot keys, grid minimum
        unsigned long long mn = ~0ull;
        // four entries per thread in flight: their list entries, then their keys
        for (uint32_t i0 = blockIdx.x * kPeelThreads + tid; i0 < na; i0 += 4 * stride) {
            uint32_t vv[4], kk[4];
            #pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + (uint64_t)u * stride;
                vv[u] = i < na ? cur[i] : 0u;
            }
            #pragma unroll
            for (int u = 0; u < 4; ++u) kk[u] = i0 + (uint64_t)u * stride < na ? kv[vv[u]] : 0u;
            #pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i0 + (uint64_t)u * stride < na) {
                    st[vv[u]] = ((unsigned long long)kUnpeeled << 32) | kk[u];
                    mn = min(mn, (unsigned long long)kk[u]);
                }
            }
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        if (lane == 0) S.red[warp] = mn;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = ~0ull;
            for (int i = 0; i < NW; ++i) b = min(b, S.red[i]);
            if (b != ~0ull) atomicMin(&pc->mn[r & 1], b);
        }
        if (!grid_barrier(pc, ctl, P, bar_target)) return;
        if (round_min && blockIdx.x == 0 && tid == 0) round_min[r] = (uint32_t)pc->mn[r & 1];
        // ---- BC: split off F; its low-degree vertices are counted here
        // F = {key * q <= min * (p + q)}, or {key < fixed_k} (then q = 1)
        const unsigned long long thr = fixed_k != kUnpeeled ? (unsigned long long)fixed_k - 1ull
                                                            : pc->mn[r & 1] * (p + q);
        // the alive list is dealt out to the blocks in chunks of 32 entries,
        // round robin, so that consecutive ids (R-MAT's high-degree vertices
        // have the smallest ids) spread over the blocks
        for (uint32_t c0 = 0; (uint64_t)(blockIdx.x + (uint64_t)P * c0) * 32 < na; c0 += NW * kSplitK) {
            // kSplitK entries per thread: their list entries, snapshot words
            // and degrees are loaded together
            uint32_t v[kSplitK];
            bool valid[kSplitK], inF[kSplitK];
            unsigned long long sv[kSplitK];
            int64_t d[kSplitK];
            #pragma unroll
            for (int k = 0; k < kSplitK; ++k) {
                const uint64_t chunk = blockIdx.x + (uint64_t)P * (c0 + warp + (uint64_t)NW * k);
                const uint64_t i = chunk * 32 + lane;
                valid[k] = i < na;
                v[k] = valid[k] ? cur[i] : 0u;
            }
            #pragma unroll
            for (int k = 0; k < kSplitK; ++k) sv[k] = valid[k] ? st[v[k]] : 0ull;
            #pragma unroll
            for (int k = 0; k < kSplitK; ++k) {
                inF[k] = valid[k] && (sv[k] & 0xffffffffull) * q <= thr;
                d[k] = 0;
                if (inF[k]) {
                    round[v[k]] = r;
                    st[v[k]] = ((unsigned long long)r << 32) | (sv[k] & 0xffffffffull);
                    d[k] = off[v[k] + 1] - off[v[k]];
                }
            }
            uint32_t ns[kSplitK];
            #pragma unroll
            for (int k = 0; k < kSplitK; ++k) {
                // arcs leaving the alive set with F (summed per block, one
                // global atomic per block and round)
                unsigned long long dsum = (unsigned long long)d[k];
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
                if (lane == 0 && dsum) atomicAdd(&S.arcs_gone, dsum);
                const bool hv = inF[k] && d[k] > kLocalDegree;
                if (hv) {
                    // heavy: global list entry (v, first chunk); its chunks are
                    // shared by all blocks after the barrier
                    A[v[k]] = 0;
                    const unsigned long long nc = (unsigned long long)((d[k] + kPeelChunk - 1) / kPeelChunk);
                    const unsigned long long old = atomicAdd(&pc->heavy[r & 1], (1ull << kHeavyShift) | nc);
                    heavy[old >> kHeavyShift] = ((unsigned long long)v[k] << kHeavyShift) | (old & kChunkMask);
                }
                const bool tv = inF[k] && d[k] <= kTinyDegree;
                const uint32_t ts = warp_claim(tv, &S.nt);
                if (tv) S.tiny[ts] = v[k];       // ts, qs < kQueueCap: drained below before they can fill
                const uint32_t qs = warp_claim(inF[k] && !hv && !tv, &S.nq);
                if (inF[k] && !hv && !tv) S.queue[qs] = v[k];
                // survivors: slots claimed in the block, then one global claim
                // per block (all warps of the grid on one counter serialise)
                ns[k] = warp_claim(valid[k] && !inF[k], &S.nsurv);
            }
            __syncthreads();
            if (tid == 0) {
                S.nbase = S.nsurv ? atomicAdd(&pc->n_next[(r + 1) & 1], S.nsurv) : 0u;
                S.nsurv = 0;
            }
            __syncthreads();
            #pragma unroll
            for (int k = 0; k < kSplitK; ++k)
                if (valid[k] && !inF[k]) nxt[S.nbase + ns[k]] = v[k];
            if (S.nq + kSplitK * kPeelThreads > (uint32_t)kQueueCap ||
                S.nt + kSplitK * kPeelThreads > (uint32_t)kQueueCap)
                drain_queue(S, off, adj, r, thr, q, st, kv, loads, A);
        }
        drain_queue(S, off, adj, r, thr, q, st, kv, loads, A);
        if (tid == 0 && S.arcs_gone) {
            atomicAdd(&pc->arcs_alive, ~S.arcs_gone + 1ull);      // subtract
            S.arcs_gone = 0;
        }
        if (!grid_barrier(pc, ctl, P, bar_target)) return;
        // ---- H: chunks of the heavier F vertices, over all blocks
        const unsigned long long hp = ld_acquire_u64(&pc->heavy[r & 1]);
        const uint32_t nh = (uint32_t)(hp >> kHeavyShift);
        if (nh > 0) {
            const unsigned long long nchunks = hp & kChunkMask;
            // the heavy list's first chunks and vertices in shared memory (the
            // queues are empty here), so that a chunk finds its vertex without
            // a dependent global load per search step; longer lists (rare)
            // are searched in global memory
            const bool local = nh <= (uint32_t)kQueueCap && nchunks <= 0xffffffffull;
            if (local && blockIdx.x < nchunks) {
                for (uint32_t i = tid; i < nh; i += kPeelThreads) {
                    const unsigned long long h = heavy[i];
                    S.queue[i] = (uint32_t)(h & kChunkMask);
                    S.tiny[i] = (uint32_t)(h >> kHeavyShift);
                }
                __syncthreads();
            }
            for (unsigned long long k = blockIdx.x; k < nchunks; k += P) {
                // the heavy entry holding chunk k: last with first chunk <= k
                uint32_t lo = 0, hi = nh - 1, v;
                unsigned long long first;
                if (local) {
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (S.queue[mid] <= k) lo = mid; else hi = mid - 1;
                    }
                    v = S.tiny[lo];
                    first = S.queue[lo];
                } else {
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if ((heavy[mid] & kChunkMask) <= k) lo = mid; else hi = mid - 1;
                    }
                    const unsigned long long h = heavy[lo];
                    v = (uint32_t)(h >> kHeavyShift);
                    first = h & kChunkMask;
                }
                const int64_t s0 = off[v] + (int64_t)(k - first) * kPeelChunk;
                const int64_t e0 = min(off[v + 1], s0 + kPeelChunk);
                uint32_t c = count_arcs(adj, s0, e0, tid, kPeelThreads, v, r, thr, q, st, kv);
                c = __reduce_add_sync(kFull, c);
                if (lane == 0 && c) {
                    atomicAdd(&A[v], c);
                    atomicAdd(&loads[v], c);
                }
            }
            if (!grid_barrier(pc, ctl, P, bar_target)) return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) pc->rounds = r;
}

// plan of the (round, id) sort: key range [0, rounds)
__global__ void k_peel_plan(Control *ctl, const PeelCtl *pc)
{
    const int tid = threadIdx.x;
    const uint32_t range = pc->rounds ? pc->rounds - 1 : 0;
    const int bits = range ? 32 - __clz(range) : 0;
    const int np = bits ? (bits + kRadixBits - 1) / kRadixBits : 1;
    for (int i = tid; i < kMaxPasses * kBuckets; i += blockDim.x) (&ctl->hist[0][0])[i] = 0;
    for (int i = tid; i < kBuckets; i += blockDim.x) ctl->asum[i] = 0;
    if (tid == 0) {
        ctl->lmin = 0;
        ctl->npass = np;
        for (int p = 0; p < kMaxPasses; ++p) ctl->shift[p] = p * kRadixBits;
        for (int p = 0; p < kMaxPasses; ++p) ctl->tile_ctr[p] = 0;
        ctl->done_ctr = 0;
        ctl->improved = 0;
        ctl->epoch += kMaxPasses;
        ctl->peel_rounds += pc->rounds;
        ctl->peel_work += pc->work;
    }
}

__global__ void k_peel_reset_width(Control *ctl) { ctl->width = 0; }

// digit histograms of the round keys and the per-digit sums of A
__global__ void k_peel_hist(const uint32_t *__restrict__ round, const uint32_t *__restrict__ A,
                            int64_t n, Control *ctl)
{
    __shared__ uint32_t h[kMaxPasses][kBuckets];
    __shared__ unsigned long long as[kBuckets];
    const int np = ctl->npass;
    uint32_t width = 0;                 // largest later-neighbour count (the trace's width)
    for (int i = threadIdx.x; i < kMaxPasses * kBuckets; i += blockDim.x) (&h[0][0])[i] = 0;
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) as[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = round[v];
        for (int p = 0; p < np; ++p) atomicAdd(&h[p][(x >> (p * kRadixBits)) & (kBuckets - 1)], 1u);
        atomicAdd(&as[(x >> ((np - 1) * kRadixBits)) & (kBuckets - 1)], (unsigned long long)A[v]);
        width = max(width, A[v]);
    }
    width = __reduce_max_sync(kFull, width);
    if ((threadIdx.x & 31) == 0 && width) atomicMax(&ctl->width, width);
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) {
        for (int p = 0; p < np; ++p)
            if (h[p][i]) atomicAdd(&ctl->hist[p][i], h[p][i]);
        if (as[i]) atomicAdd(&ctl->asum[i], as[i]);
    }
}

__global__ void k_peel_snapshot(const uint32_t *__restrict__ round, uint32_t *__restrict__ best,
                                int64_t n, const Control *ctl)
{
    if (!ctl->improved) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        best[v] = round[v];
}

void peel_free(PeelBufs &pb, cudaStream_t s)
{
    if (pb.mem) cudaFreeAsync(pb.mem, s);
    pb.mem = nullptr;
}

static int g_peel_blocks_per_sm = -1;
static std::once_flag g_peel_once;

int peel_run(cudaStream_t s, const GraphDev &g, RunBufs &b, PeelBufs &pb, bool &pb_ready,
             int sm_count, int max_blocks, int T, int64_t p, int64_t q, int *launches, std::string &err)
{
    const int64_t n = g.n;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sz4 = al(4 * (size_t)n), sz8 = al(8 * (size_t)n), sz_pc = al(sizeof(PeelCtl));
    if (!pb_ready) {
        const size_t total = 4 * sz4 + 2 * sz8 + sz_pc;
        cudaError_t e = dev_malloc(&pb.mem, total, s);
        if (e != cudaSuccess) {
            err = std::string("peel buffers: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DSG_ERR_NOMEM : DSG_ERR_CUDA;
        }
        cudaMemsetAsync(pb.mem, 0, total, s);
        pb.bytes = total;
        pb_ready = true;
    }
    char *m = (char *)pb.mem;
    uint32_t *kv = (uint32_t *)m;
    uint32_t *round = (uint32_t *)(m + sz4);
    uint32_t *list0 = (uint32_t *)(m + 2 * sz4);
    uint32_t *list1 = (uint32_t *)(m + 3 * sz4);
    unsigned long long *st = (unsigned long long *)(m + 4 * sz4);
    unsigned long long *heavy = (unsigned long long *)(m + 4 * sz4 + sz8);
    PeelCtl *pc = (PeelCtl *)(m + 4 * sz4 + 2 * sz8);

    std::call_once(g_peel_once, [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peel, kPeelThreads, 0);
        g_peel_blocks_per_sm = nb >= 2 ? 2 : (nb > 0 ? 1 : 0);
    });
    if (g_peel_blocks_per_sm < 1) {
        err = "the peel kernel cannot be resident";
        return DSG_ERR_CUDA;
    }
    // blocks: the resident blocks of at most max_blocks SMs (two per SM),
    // and no more than the vertices and arcs need
    const int grid = (int)imin64(imin64((int64_t)sm_count, max_blocks) * g_peel_blocks_per_sm, peel_blocks((uint64_t)n, (uint64_t)g.arcs));
    const int igrid = (int)imin64((n + 255) / 256, (int64_t)sm_count * 8);
    int nl = 0;
    for (int t = 1; t <= T; ++t) {
        k_peel_reset_width<<<1, 1, 0, s>>>(b.ctl);
        k_peel_init<<<igrid, 256, 0, s>>>(g.off, b.loads, n, g.arcs, kv, round, list0, pc);
        const int64_t *off = g.off;
        const int32_t *adj = g.adj;
        uint32_t *loads = b.loads, *A = b.A;
        uint64_t pp = (uint64_t)p, qq = (uint64_t)q;
        int64_t nn = n;
        Control *ctl = b.ctl;
        uint32_t *no_rmin = nullptr;
        uint32_t no_fixed = kUnpeeled;
        void *args[] = {(void *)&off, (void *)&adj, (void *)&nn, (void *)&loads, (void *)&A,
                        (void *)&kv, (void *)&st, (void *)&round, (void *)&list0, (void *)&list1,
                        (void *)&heavy, (void *)&pp, (void *)&qq, (void *)&pc, (void *)&ctl, (void *)&no_rmin,
                        (void *)&no_fixed};
        cudaError_t e = cudaLaunchCooperativeKernel((void *)k_peel, grid, kPeelThreads, args, 0, s);
        if (e != cudaSuccess) {
            err = std::string("cooperative peel launch: ") + cudaGetErrorString(e);
            return DSG_ERR_CUDA;
        }
        k_peel_plan<<<1, 256, 0, s>>>(b.ctl, pc);
        k_peel_hist<<<igrid, 256, 0, s>>>(round, b.A, n, b.ctl);
        e = launch_radix_passes(g, b, t, s, round, false);
        if (e != cudaSuccess) {
            err = std::string("radix pass: ") + cudaGetErrorString(e);
            return DSG_ERR_CUDA;
        }
        k_peel_snapshot<<<igrid, 256, 0, s>>>(round, b.best_loads, n, b.ctl);
        nl += 6 + kMaxPasses;
    }
    if (launches) *launches += nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("peel: ") + cudaGetErrorString(e);
        return DSG_ERR_CUDA;
    }
    return DSG_OK;
}

// ---- coreness (Sec. 2, Definition of core number): the round peel with
// eps = 0 from zero loads peels, each round, the alive vertices of minimum
// induced degree; the core number of a vertex is the largest round minimum
// up to its round.

// inclusive prefix maximum of x[0..R) (single block)
__global__ void k_prefix_max(uint32_t *x, int64_t R)
{
    __shared__ uint32_t part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (R + blockDim.x - 1) / blockDim.x;
    const int64_t b = tid * per, e = imin64(R, b + per);
    uint32_t mx = 0;
    for (int64_t i = b; i < e; ++i) mx = max(mx, x[i]);
    part[tid] = mx;
    __syncthreads();
    if (tid == 0)
        for (int i = 1; i < (int)blockDim.x; ++i) part[i] = max(part[i], part[i - 1]);
    __syncthreads();
    uint32_t run = tid ? part[tid - 1] : 0u;
    for (int64_t i = b; i < e; ++i) {
        run = max(run, x[i]);
        x[i] = run;
    }
}

__global__ void k_core_assign(const uint32_t *__restrict__ round, const uint32_t *__restrict__ cmax, int64_t n,
                              int32_t *core)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        core[v] = (int32_t)cmax[round[v]];
}

int coreness_run(cudaStream_t s, const GraphDev &g, Control *ctl, int sm_count, int32_t *core, int64_t *kmax,
                 std::string &err)
{
    const int64_t n = g.n;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sz4 = al(4 * (size_t)n), sz8 = al(8 * (size_t)n), sz_pc = al(sizeof(PeelCtl));
    const size_t total = 7 * sz4 + 2 * sz8 + sz_pc;
    void *mem = nullptr;
    cudaError_t e = dev_malloc(&mem, total, s);
    if (e != cudaSuccess) {
        err = std::string("coreness buffers: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DSG_ERR_NOMEM : DSG_ERR_CUDA;
    }
    cudaMemsetAsync(mem, 0, total, s);
    char *m = (char *)mem;
    uint32_t *kv = (uint32_t *)m, *round = (uint32_t *)(m + sz4), *list0 = (uint32_t *)(m + 2 * sz4);
    uint32_t *list1 = (uint32_t *)(m + 3 * sz4), *zl = (uint32_t *)(m + 4 * sz4), *A = (uint32_t *)(m + 5 * sz4);
    uint32_t *rmin = (uint32_t *)(m + 6 * sz4);
    unsigned long long *st = (unsigned long long *)(m + 7 * sz4);
    unsigned long long *heavy = (unsigned long long *)(m + 7 * sz4 + sz8);
    PeelCtl *pc = (PeelCtl *)(m + 7 * sz4 + 2 * sz8);
    std::call_once(g_peel_once, [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peel, kPeelThreads, 0);
        g_peel_blocks_per_sm = nb >= 2 ? 2 : (nb > 0 ? 1 : 0);
    });
    if (g_peel_blocks_per_sm < 1) {
        cudaFreeAsync(mem, s);
        err = "the peel kernel cannot be resident";
        return DSG_ERR_CUDA;
    }
    const int grid = (int)imin64((int64_t)sm_count * g_peel_blocks_per_sm, peel_blocks((uint64_t)n, (uint64_t)g.arcs));
    const int igrid = (int)imin64((n + 255) / 256, (int64_t)sm_count * 8);
    // a failure status or test knob left by an earlier run does not carry over
    cudaMemsetAsync(&ctl->err, 0, 16, s);
    k_peel_init<<<igrid, 256, 0, s>>>(g.off, zl, n, g.arcs, kv, round, list0, pc);
    const int64_t *off = g.off;
    const int32_t *adj = g.adj;
    uint64_t pp = 0, qq = 1;
    int64_t nn = n;
    uint32_t no_fixed = kUnpeeled;
    void *args[] = {(void *)&off, (void *)&adj, (void *)&nn, (void *)&zl, (void *)&A, (void *)&kv, (void *)&st,
                    (void *)&round, (void *)&list0, (void *)&list1, (void *)&heavy, (void *)&pp, (void *)&qq,
                    (void *)&pc, (void *)&ctl, (void *)&rmin, (void *)&no_fixed};
    e = cudaLaunchCooperativeKernel((void *)k_peel, grid, kPeelThreads, args, 0, s);
    uint32_t rounds = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rounds, &pc->rounds, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && rounds > 0) {
        k_prefix_max<<<1, 1024, 0, s>>>(rmin, rounds);
        k_core_assign<<<igrid, 256, 0, s>>>(round, rmin, n, core);
        uint32_t km = 0;
        cudaMemcpyAsync(&km, rmin + rounds - 1, 4, cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        *kmax = km;
    }
    int cerr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cerr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && cerr) {
        cudaFreeAsync(mem, s);
        err = "coreness: a bounded wait gave up";
        return cerr;
    }
    cudaFreeAsync(mem, s);
    if (e != cudaSuccess) {
        err = std::string("coreness: ") + cudaGetErrorString(e);
        return DSG_ERR_CUDA;
    }
    return DSG_OK;
}

// ---- the k-core by deletion (Sec. 2, Definition of k-core): rounds that
// remove every alive vertex of induced degree < k at once, until a round
// removes nothing; keep[v] = k for the survivors, 0 for the others.
__global__ void k_kcore_mark(const uint32_t *__restrict__ round, int64_t n, int32_t k, int32_t *keep)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = (!round || round[v] == kUnpeeled) ? k : 0;
}

KCoreBufs::~KCoreBufs() = default;

int kcore_run(cudaStream_t s, const GraphDev &g, Control *ctl, int sm_count, KCoreBufs &kb, int32_t k,
              int32_t *keep, int64_t *survivors, std::string &err)
{
    const int64_t n = g.n;
    const int igrid0 = (int)imax64(1, imin64((n + 255) / 256, (int64_t)sm_count * 8));
    if (k <= 0) {                          // the 0-core is the whole graph
        k_kcore_mark<<<igrid0, 256, 0, s>>>(nullptr, n, 0, keep);
        *survivors = n;
        return cudaGetLastError() == cudaSuccess ? DSG_OK : DSG_ERR_CUDA;
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sz4 = al(4 * (size_t)n), sz8 = al(8 * (size_t)n), sz_pc = al(sizeof(PeelCtl));
    const size_t total = 6 * sz4 + 2 * sz8 + sz_pc;
    cudaError_t e;
    if (kb.bytes < total) {
        if (kb.mem) cudaFreeAsync(kb.mem, s);
        kb.mem = nullptr;
        kb.bytes = 0;
        if ((e = dev_malloc(&kb.mem, total, s)) != cudaSuccess) {
            err = std::string("k-core buffers: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DSG_ERR_NOMEM : DSG_ERR_CUDA;
        }
        kb.bytes = total;
    }
    char *m = (char *)kb.mem;
    uint32_t *kv = (uint32_t *)m, *round = (uint32_t *)(m + sz4), *list0 = (uint32_t *)(m + 2 * sz4);
    uint32_t *list1 = (uint32_t *)(m + 3 * sz4), *zl = (uint32_t *)(m + 4 * sz4), *A = (uint32_t *)(m + 5 * sz4);
    unsigned long long *st = (unsigned long long *)(m + 6 * sz4);
    unsigned long long *heavy = (unsigned long long *)(m + 6 * sz4 + sz8);
    PeelCtl *pc = (PeelCtl *)(m + 6 * sz4 + 2 * sz8);
    cudaMemsetAsync(zl, 0, 4 * (size_t)n, s);
    std::call_once(g_peel_once, [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peel, kPeelThreads, 0);
        g_peel_blocks_per_sm = nb >= 2 ? 2 : (nb > 0 ? 1 : 0);
    });
    if (g_peel_blocks_per_sm < 1) {
        err = "the peel kernel cannot be resident";
        return DSG_ERR_CUDA;
    }
    const int grid = (int)imin64((int64_t)sm_count * g_peel_blocks_per_sm, peel_blocks((uint64_t)n, (uint64_t)g.arcs));
    const int igrid = (int)imin64((n + 255) / 256, (int64_t)sm_count * 8);
    // a failure status or test knob left by an earlier run does not carry over
    cudaMemsetAsync(&ctl->err, 0, 16, s);
    k_peel_init<<<igrid, 256, 0, s>>>(g.off, zl, n, g.arcs, kv, round, list0, pc);
    const int64_t *off = g.off;
    const int32_t *adj = g.adj;
    uint64_t pp = 0, qq = 1;
    int64_t nn = n;
    uint32_t *no_rmin = nullptr;
    uint32_t fk = (uint32_t)k;
    void *args[] = {(void *)&off, (void *)&adj, (void *)&nn, (void *)&zl, (void *)&A, (void *)&kv, (void *)&st,
                    (void *)&round, (void *)&list0, (void *)&list1, (void *)&heavy, (void *)&pp, (void *)&qq,
                    (void *)&pc, (void *)&ctl, (void *)&no_rmin, (void *)&fk};
    e = cudaLaunchCooperativeKernel((void *)k_peel, grid, kPeelThreads, args, 0, s);
    if (e == cudaSuccess) k_kcore_mark<<<igrid, 256, 0, s>>>(round, n, k, keep);
    uint32_t alive[2] = {0, 0};
    int cerr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(alive, pc->n_next, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cerr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    uint32_t rounds = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rounds, &pc->rounds, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        err = std::string("k-core: ") + cudaGetErrorString(e);
        return DSG_ERR_CUDA;
    }
    if (cerr) {
        err = "k-core: a bounded wait gave up";
        return cerr;
    }
    // the survivors are the alive list of the last round
    *survivors = alive[rounds & 1];
    return DSG_OK;
}

void kcore_free(KCoreBufs &kb, cudaStream_t s)
{
    if (kb.mem) cudaFreeAsync(kb.mem, s);
    kb.mem = nullptr;
    kb.bytes = 0;
}

}  // namespace dsg
