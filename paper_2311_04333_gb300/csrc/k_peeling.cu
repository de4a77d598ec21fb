// k_peeling.cu -- PaRGreedy++ refine step (arXiv 2311.04333, Sec. 3.3
// "ParallelGreedy++"): the ordering comes from bucketed peeling by the key
// l(v) + deg_H(v) with H reset to G each iteration.  Each round peels every
// alive vertex whose key is within a factor (1 + p/q) of the round's minimum
// key (key*q <= min*(p+q)), all at once; the degree decrements they cause are
// applied only after the round's set is fixed.  The order is (round, id).
//
// One cooperative persistent kernel runs all rounds of an iteration; each
// round has three phases separated by bounded grid barriers:
//   A: key of every alive vertex, grid minimum;
//   B: split the alive list into the round's set F (round[v] = r) and the
//      next alive list;
//   C: for v in F, count its later neighbours (alive ones, and same-round
//      ones with a larger id) -> A[v], l(v) += A[v], and decrement deg_H of
//      the alive neighbours.
// The densest suffix of the (round, id) order then reuses the radix passes
// of the sorting path with key = round and value = A (Alg. 3 lines 4-7).
#include <mutex>

#include "common.cuh"
#include "dsg.h"
#include "peeling.h"

namespace dsg {

constexpr uint32_t kUnpeeled = 0xffffffffu;
constexpr int kPeelThreads = 256;
constexpr int64_t kBigDegree = 2048;     // F vertices above this use a whole block

struct PeelCtl {
    unsigned long long mn[2];   // round minimum key, by round parity
    uint32_t n_next[2];         // alive-list sizes, by round parity
    uint32_t n_fs[2], n_fb[2];  // small / big F sizes, by round parity
    uint32_t rounds;
    uint32_t bar_count, bar_gen;
    uint32_t abort;
    unsigned long long work;    // sum over rounds of the alive-list size
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded grid barrier (all blocks are co-resident: cooperative launch)
__device__ __forceinline__ bool grid_barrier(PeelCtl *pc, Control *ctl, uint32_t nblocks)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t gen = ld_acquire_u32(&pc->bar_gen);
        __threadfence();
        if (atomicAdd(&pc->bar_count, 1u) == nblocks - 1) {
            pc->bar_count = 0;
            __threadfence();
            atomicAdd(&pc->bar_gen, 1u);
        } else {
            uint32_t polls = 0, ns = 32;
            while (ld_acquire_u32(&pc->bar_gen) == gen) {
                if (ld_acquire_u32(&pc->abort) || ++polls > kSpinLimit) {
                    atomicExch(&pc->abort, 1u);
                    set_error(ctl, DSG_ERR_TIMEOUT, 400);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
        }
        __threadfence();
        if (ld_acquire_u32(&pc->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void k_peel_init(const int64_t *__restrict__ off, int64_t n, int32_t *deg,
                            uint32_t *round, uint32_t *list0, PeelCtl *pc)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        deg[v] = (int32_t)(off[v + 1] - off[v]);
        round[v] = kUnpeeled;
        list0[v] = (uint32_t)v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pc->mn[0] = pc->mn[1] = ~0ull;
        pc->n_next[0] = (uint32_t)n;
        pc->n_next[1] = 0;
        pc->n_fs[0] = pc->n_fs[1] = 0;
        pc->n_fb[0] = pc->n_fb[1] = 0;
        pc->rounds = 0;
        pc->bar_count = 0;
        pc->abort = 0;
        pc->work = 0;
    }
}

// warp-aggregated append of v (if pred) to list[] through counter *cnt
__device__ __forceinline__ void warp_append(bool pred, uint32_t v, uint32_t *list, uint32_t *cnt)
{
    const uint32_t m = __ballot_sync(kFull, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) list[base + __popc(m & lanemask_lt())] = v;
}

__global__ void __launch_bounds__(kPeelThreads)
k_peel(const int64_t *__restrict__ off, const int32_t *__restrict__ adj, int64_t n,
       uint32_t *loads, uint32_t *A, int32_t *deg, uint32_t *round, uint32_t *list0,
       uint32_t *list1, uint32_t *flist, unsigned long long *keybuf, uint64_t p, uint64_t q,
       PeelCtl *pc, Control *ctl)
{
    __shared__ unsigned long long s_min[kPeelThreads / 32];
    __shared__ uint32_t s_cnt[kPeelThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nb = gridDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + tid;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gtid >> 5, gwarps = gthreads >> 5;
    uint32_t width = 0;
    uint32_t r = 0;
    for (;; ++r) {
        const uint32_t na = ld_acquire_u32(&pc->n_next[r & 1]);
        if (na == 0) break;
        uint32_t *cur = (r & 1) ? list1 : list0;
        uint32_t *nxt = (r & 1) ? list0 : list1;
        if (blockIdx.x == 0 && tid == 0) {
            pc->n_next[(r + 1) & 1] = 0;
            pc->mn[(r + 1) & 1] = ~0ull;
            pc->n_fs[(r + 1) & 1] = 0;
            pc->n_fb[(r + 1) & 1] = 0;
            pc->work += na;
        }
        // ---- phase A: keys and their minimum
        unsigned long long mn = ~0ull;
        for (int64_t i = gtid; i < na; i += gthreads) {
            const uint32_t v = cur[i];
            const unsigned long long key = (unsigned long long)loads[v] + (unsigned long long)deg[v];
            keybuf[i] = key;
            mn = min(mn, key);
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        if (lane == 0) s_min[warp] = mn;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = ~0ull;
            for (int i = 0; i < kPeelThreads / 32; ++i) b = min(b, s_min[i]);
            if (b != ~0ull) atomicMin(&pc->mn[r & 1], b);
        }
        if (!grid_barrier(pc, ctl, nb)) return;
        // ---- phase B: the round's set F = {key*q <= min*(p+q)}
        const unsigned long long thr = pc->mn[r & 1] * (p + q);
        for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < na; i0 += gthreads) {
            const int64_t i = i0 + tid;
            const bool valid = i < na;
            uint32_t v = 0;
            bool inF = false;
            if (valid) {
                v = cur[i];
                inF = keybuf[i] * q <= thr;
                if (inF) round[v] = r;
            }
            const bool big = inF && (off[v + 1] - off[v] > kBigDegree);
            warp_append(inF && !big, v, flist, &pc->n_fs[r & 1]);
            // big ones fill flist from the back
            const uint32_t mb = __ballot_sync(kFull, big);
            if (mb) {
                const int leader = __ffs(mb) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(&pc->n_fb[r & 1], (uint32_t)__popc(mb));
                base = __shfl_sync(kFull, base, leader);
                if (big) flist[n - 1 - (base + __popc(mb & lanemask_lt()))] = v;
            }
            warp_append(valid && !inF, v, nxt, &pc->n_next[(r + 1) & 1]);
        }
        if (!grid_barrier(pc, ctl, nb)) return;
        // ---- phase C: later-neighbour counts and delayed degree decrements
        const uint32_t nfs = pc->n_fs[r & 1], nfb = pc->n_fb[r & 1];
        for (int64_t f = gwarp; f < nfs; f += gwarps) {
            const uint32_t v = flist[f];
            const int64_t s = off[v], e = off[v + 1];
            uint32_t c = 0;
            for (int64_t j = s + lane; j < e; j += 32) {
                const uint32_t w = (uint32_t)adj[j];
                const uint32_t rw = round[w];
                if (rw == kUnpeeled) {
                    ++c;
                    atomicSub(&deg[w], 1);
                } else if (rw == r && w > v) {
                    ++c;
                }
            }
            c = __reduce_add_sync(kFull, c);
            if (lane == 0) {
                A[v] = c;
                loads[v] += c;
                width = max(width, c);
            }
        }
        for (int64_t f = blockIdx.x; f < nfb; f += gridDim.x) {
            const uint32_t v = flist[n - 1 - f];
            const int64_t s = off[v], e = off[v + 1];
            uint32_t c = 0;
            for (int64_t j = s + tid; j < e; j += kPeelThreads) {
                const uint32_t w = (uint32_t)adj[j];
                const uint32_t rw = round[w];
                if (rw == kUnpeeled) {
                    ++c;
                    atomicSub(&deg[w], 1);
                } else if (rw == r && w > v) {
                    ++c;
                }
            }
            c = __reduce_add_sync(kFull, c);
            if (lane == 0) s_cnt[warp] = c;
            __syncthreads();
            if (tid == 0) {
                uint32_t tot = 0;
                for (int i = 0; i < kPeelThreads / 32; ++i) tot += s_cnt[i];
                A[v] = tot;
                loads[v] += tot;
                width = max(width, tot);
            }
            __syncthreads();
        }
        if (!grid_barrier(pc, ctl, nb)) return;
    }
    width = __reduce_max_sync(kFull, width);
    if (lane == 0 && width) atomicMax(&ctl->width, width);
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
    for (int i = threadIdx.x; i < kMaxPasses * kBuckets; i += blockDim.x) (&h[0][0])[i] = 0;
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) as[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = round[v];
        for (int p = 0; p < np; ++p) atomicAdd(&h[p][(x >> (p * kRadixBits)) & (kBuckets - 1)], 1u);
        atomicAdd(&as[(x >> ((np - 1) * kRadixBits)) & (kBuckets - 1)], (unsigned long long)A[v]);
    }
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
             int sm_count, int T, int64_t p, int64_t q, int *launches, std::string &err)
{
    const int64_t n = g.n;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sz_deg = al(4 * (size_t)n), sz_round = al(4 * (size_t)n), sz_list = al(4 * (size_t)n);
    const size_t sz_key = al(8 * (size_t)n), sz_pc = al(sizeof(PeelCtl));
    if (!pb_ready) {
        const size_t total = sz_deg + sz_round + 3 * sz_list + sz_key + sz_pc;
        cudaError_t e = cudaMallocAsync(&pb.mem, total, s);
        if (e != cudaSuccess) {
            err = std::string("peel buffers: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DSG_ERR_NOMEM : DSG_ERR_CUDA;
        }
        cudaMemsetAsync(pb.mem, 0, total, s);
        pb.bytes = total;
        pb_ready = true;
    }
    char *m = (char *)pb.mem;
    int32_t *deg = (int32_t *)m;
    uint32_t *round = (uint32_t *)(m + sz_deg);
    uint32_t *list0 = (uint32_t *)(m + sz_deg + sz_round);
    uint32_t *list1 = (uint32_t *)(m + sz_deg + sz_round + sz_list);
    uint32_t *flist = (uint32_t *)(m + sz_deg + sz_round + 2 * sz_list);
    unsigned long long *keybuf = (unsigned long long *)(m + sz_deg + sz_round + 3 * sz_list);
    PeelCtl *pc = (PeelCtl *)(m + sz_deg + sz_round + 3 * sz_list + sz_key);

    std::call_once(g_peel_once, [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peel, kPeelThreads, 0);
        g_peel_blocks_per_sm = nb > 0 ? (nb < 4 ? nb : 4) : 1;
    });
    const int grid = sm_count * g_peel_blocks_per_sm;
    const int igrid = (int)imin64((n + 255) / 256, (int64_t)sm_count * 8);
    int nl = 0;
    for (int t = 1; t <= T; ++t) {
        k_peel_reset_width<<<1, 1, 0, s>>>(b.ctl);
        k_peel_init<<<igrid, 256, 0, s>>>(g.off, n, deg, round, list0, pc);
        const int64_t *off = g.off;
        const int32_t *adj = g.adj;
        uint32_t *loads = b.loads, *A = b.A;
        uint64_t pp = (uint64_t)p, qq = (uint64_t)q;
        int64_t nn = n;
        Control *ctl = b.ctl;
        void *args[] = {(void *)&off, (void *)&adj, (void *)&nn, (void *)&loads, (void *)&A,
                        (void *)&deg, (void *)&round, (void *)&list0, (void *)&list1,
                        (void *)&flist, (void *)&keybuf, (void *)&pp, (void *)&qq, (void *)&pc,
                        (void *)&ctl};
        cudaError_t e = cudaLaunchCooperativeKernel((void *)k_peel, grid, kPeelThreads, args, 0, s);
        if (e != cudaSuccess) {
            err = std::string("cooperative peel launch: ") + cudaGetErrorString(e);
            return DSG_ERR_CUDA;
        }
        k_peel_plan<<<1, 256, 0, s>>>(b.ctl, pc);
        k_peel_hist<<<igrid, 256, 0, s>>>(round, b.A, n, b.ctl);
        for (int k = 0; k < kMaxPasses; ++k) {
            e = launch_radix_pass(g, b, k, t, s, round, false);
            if (e != cudaSuccess) {
                err = std::string("radix pass: ") + cudaGetErrorString(e);
                return DSG_ERR_CUDA;
            }
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

}  // namespace dsg
