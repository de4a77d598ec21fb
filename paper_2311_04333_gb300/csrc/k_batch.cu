// k_batch.cu -- batched refine step (arXiv 2311.04333, Sec. 3.2-3.3 with
// Alg. 3), PaRSorting++ or PaRGreedy++, for many small graphs packed into one
// segmented CSR.  One persistent launch: every block takes whole graphs from
// an atomic queue (largest first) and runs all T iterations of a graph by
// itself:
//   order      PaRSorting++: edge scan A[u] = #{w in N(u) : (l[w], w) >
//              (l[u], u)} (warp per vertex), keys = loads;
//              PaRGreedy++: rounds of bucketed peeling with the count of
//              later neighbours fused (block_peel), keys = rounds
//   sort       stable LSD radix sort of the ids by key - min key (8-bit
//              digits); the block's warps own contiguous segments: count,
//              scan in (digit, warp) order, ranked scatter
//   suffix     B[i] = sum_{j >= i} A[v_j]; first maximum of B[i] / (n - i)
//              (Alg. 3, suffix densities); strict update of the graph's best (Alg. 2)
//   loads      l += A (Alg. 3, load update; PaRGreedy++ adds each count as its
//              vertex is peeled)
// and finally extracts the best vertex set.  Graph g owns vertices
// [vbase[g], vbase[g+1]) and arcs [off[vbase[g]], off[vbase[g+1]]) of the
// packed arrays; adjacency entries are local ids.
#include "batch.h"
#include "dsg.h"
#include "common.cuh"

namespace dsg {
namespace {

template <int NT>
struct BatchSmem {
    uint32_t cnt[NT / 32][kBuckets];     // per-warp digit counts, then write cursors
    uint32_t base[kBuckets];
    unsigned long long red[33];
    Candidate cred[32];
    uint32_t wred[32];
    uint32_t graph;
    uint32_t na_next, nf, nbig;          // PaRGreedy++ round counters
    uint32_t big[64];                    // the round's F vertices of high degree
};

template <int NT>
__device__ __forceinline__ uint32_t block_reduce_u32(uint32_t x, bool is_max, BatchSmem<NT> &S)
{
    x = is_max ? __reduce_max_sync(kFull, x) : __reduce_min_sync(kFull, x);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.wred[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t r = is_max ? 0u : 0xffffffffu;
    for (int i = 0; i < NT / 32; ++i) r = is_max ? max(r, S.wred[i]) : min(r, S.wred[i]);
    __syncthreads();
    return r;
}

// lanes (among the valid ones) holding the same 8-bit digit (invalid lanes
// match only themselves)
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid)
{
    const uint32_t peers = __match_any_sync(kFull, valid ? d : (uint32_t)kBuckets + (threadIdx.x & 31));
    return valid ? peers : 0u;
}

// One stable LSD pass over elements 0..n-1: (kin, iin) -> (kout, iout) by
// the digit (key >> shift) & 255.  kin == nullptr: keys are L[i] - lmin and
// ids are i (the loads read in id order).
template <int NT>
__device__ void block_radix_pass(const uint32_t *kin, const uint32_t *iin, const uint32_t *L,
                                 uint32_t lmin, uint32_t *kout, uint32_t *iout, uint32_t n,
                                 int shift, BatchSmem<NT> &S)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t seg = (n + NW - 1) / NW;
    const uint32_t b0 = min(n, warp * seg), b1 = min(n, b0 + seg);
    for (int i = threadIdx.x; i < NW * kBuckets; i += NT) (&S.cnt[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t r = b0; r < b1; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < b1;
        const uint32_t key = valid ? (kin ? kin[i] : L[i] - lmin) : 0u;
        const uint32_t d = (key >> shift) & (kBuckets - 1);
        const uint32_t peers = digit_peers(d, valid);
        if (valid && (peers >> lane) == 1u) S.cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, and the digit's total
    uint32_t total = 0;
    if (threadIdx.x < kBuckets) {
        const int d = threadIdx.x;
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = S.cnt[w][d];
            S.cnt[w][d] = total;
            total += c;
        }
    }
    uint64_t all;
    const uint64_t ex = block_excl_sum_u64(threadIdx.x < kBuckets ? total : 0u, S.red, &all);
    if (threadIdx.x < kBuckets) S.base[threadIdx.x] = (uint32_t)ex;
    __syncthreads();
    for (int i = threadIdx.x; i < NW * kBuckets; i += NT) (&S.cnt[0][0])[i] += S.base[i % kBuckets];
    __syncthreads();
    // ranked scatter of the warp's segment, in order
    for (uint32_t r = b0; r < b1; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < b1;
        const uint32_t key = valid ? (kin ? kin[i] : L[i] - lmin) : 0u;
        const uint32_t id = valid ? (iin ? iin[i] : i) : 0u;
        const uint32_t d = (key >> shift) & (kBuckets - 1);
        const uint32_t peers = digit_peers(d, valid);
        uint32_t cur = 0;
        if (valid) cur = S.cnt[warp][d];
        __syncwarp();
        if (valid) {
            const uint32_t p = cur + __popc(peers & lanemask_lt());
            kout[p] = key;
            iout[p] = id;
            if ((peers >> lane) == 1u) S.cnt[warp][d] = cur + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
}

constexpr uint32_t kNotPeeled = 0xffffffffu;
constexpr int kScanK = 8;            // positions per thread of the suffix scan
constexpr int kBigCap = 64;

template <int NT>
__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long x, BatchSmem<NT> &S)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(kFull, x, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned long long r = ~0ull;
    for (int i = 0; i < NT / 32; ++i) r = min(r, S.red[i]);
    __syncthreads();
    return r;
}

// warp-aggregated slot claim on a shared counter (all lanes call it)
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

// PaRGreedy++ ordering of one graph by one block (Sec. 3.3): rounds peel
// F = {alive v : (l(v) + deg_H(v)) * q <= min * (p + q)}; the decrements of
// deg_H caused by F are applied after F is fixed.  Fused with the count of
// later neighbours in the (round, id) order: A[v] = alive neighbours not in
// F, plus neighbours in F with a larger id; l(v) += A[v] (Alg. 3, load update).
// R[v] receives v's round; returns the number of rounds.
template <int NT>
__device__ uint32_t block_peel(const int64_t *off, const int32_t *adj, uint32_t n, uint64_t p, uint64_t q,
                               uint32_t *L, uint32_t *A, uint32_t *R, uint32_t *deg, uint32_t *cur,
                               uint32_t *nxt, uint32_t &width, int64_t block_deg, BatchSmem<NT> &S)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t v = threadIdx.x; v < n; v += NT) {
        deg[v] = (uint32_t)(off[v + 1] - off[v]);
        R[v] = kNotPeeled;
        cur[v] = v;
    }
    uint32_t na = n, r = 0;
    for (; na > 0; ++r) {
        // keys of the alive vertices and their minimum
        unsigned long long mn = ~0ull;
        for (uint32_t i = threadIdx.x; i < na; i += NT) {
            const uint32_t v = cur[i];
            mn = min(mn, (unsigned long long)L[v] + deg[v]);
        }
        if (threadIdx.x == 0) {
            S.na_next = 0;
            S.nf = 0;
            S.nbig = 0;
        }
        mn = block_min_u64<NT>(mn, S);
        const unsigned long long thr = mn * (p + q);
        // the round's set F (back of nxt, or S.big) and the survivors (front of nxt)
        for (uint32_t i0 = warp * 32; i0 < na; i0 += NT) {
            const uint32_t i = i0 + lane;
            const bool valid = i < na;
            const uint32_t v = valid ? cur[i] : 0u;
            const bool inF = valid && ((unsigned long long)L[v] + deg[v]) * q <= thr;
            if (inF) R[v] = r;
            const bool big = inF && off[v + 1] - off[v] > block_deg;
            const uint32_t bs = warp_claim(big, &S.nbig);
            const bool stored = big && bs < (uint32_t)kBigCap;
            if (stored) S.big[bs] = v;
            const uint32_t fs = warp_claim(inF && !stored, &S.nf);
            if (inF && !stored) nxt[n - 1 - fs] = v;
            const uint32_t ns = warp_claim(valid && !inF, &S.na_next);
            if (valid && !inF) nxt[ns] = v;
        }
        __syncthreads();
        const uint32_t nf = S.nf, nbig = min(S.nbig, (uint32_t)kBigCap), na_next = S.na_next;
        for (uint32_t j = warp; j < nf; j += NW) {
            const uint32_t v = nxt[n - 1 - j];
            uint32_t c = 0;
            for (int64_t k = off[v] + lane; k < off[v + 1]; k += 32) {
                const uint32_t w = (uint32_t)adj[k];
                const uint32_t rw = R[w];
                if (rw == kNotPeeled) {
                    ++c;
                    atomicSub(&deg[w], 1u);
                } else if (rw == r && w > v) {
                    ++c;
                }
            }
            c = __reduce_add_sync(kFull, c);
            if (lane == 0) {
                A[v] = c;
                L[v] += c;
            }
            width = max(width, c);
        }
        for (uint32_t b = 0; b < nbig; ++b) {
            const uint32_t v = S.big[b];
            uint32_t c = 0;
            for (int64_t k = off[v] + threadIdx.x; k < off[v + 1]; k += NT) {
                const uint32_t w = (uint32_t)adj[k];
                const uint32_t rw = R[w];
                if (rw == kNotPeeled) {
                    ++c;
                    atomicSub(&deg[w], 1u);
                } else if (rw == r && w > v) {
                    ++c;
                }
            }
            uint64_t tot;
            block_excl_sum_u64(c, S.red, &tot);
            if (threadIdx.x == 0) {
                A[v] = (uint32_t)tot;
                L[v] += (uint32_t)tot;
            }
            width = max(width, (uint32_t)tot);
        }
        __syncthreads();
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
        na = na_next;
    }
    return r;
}

template <int NT, bool PEEL>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_batch_run(BatchDev B, uint32_t *graph_ctr)
{
    __shared__ BatchSmem<NT> S;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) S.graph = atomicAdd(graph_ctr, 1u);
        __syncthreads();
        const uint32_t qi = S.graph;
        __syncthreads();
        if (qi >= (uint32_t)B.G) break;
        const int g = B.order[qi];
        const int64_t vb = B.vbase[g];
        const uint32_t n = (uint32_t)(B.vbase[g + 1] - vb);
        const int64_t *off = B.off + vb;          // global arc indices
        const int32_t *adj = B.adj;
        const int64_t m = (off[n] - off[0]) / 2;
        const int T = B.T[g];
        uint32_t *L = B.loads + vb;
        uint32_t *A = B.A + vb;
        uint32_t *K0 = B.keys + 2 * vb, *K1 = K0 + n;
        uint32_t *I0 = B.ids + 2 * vb, *I1 = I0 + n;
        uint32_t *BL = B.best_loads + vb;
        uint32_t *R = B.round + vb;
        const uint64_t pp = PEEL ? (uint64_t)B.pq[2 * g] : 0u, qq = PEEL ? (uint64_t)B.pq[2 * g + 1] : 1u;
        for (uint32_t v = threadIdx.x; v < n; v += NT) L[v] = B.init ? (uint32_t)B.init[vb + v] : 0u;
        int64_t best_e = m, best_v = n, best_pos = 0;
        uint32_t best_key = 0, best_id = 0;
        int best_iter = 0;
        __syncthreads();
        for (int t = 1; t <= T; ++t) {
            uint32_t width = 0, lmin = 0, range = 0;
            const uint32_t *src = L;              // sort keys: loads, or rounds
            if (PEEL) {
                // ---- ordering by rounds of peeling, later-neighbour counts fused
                const uint32_t rounds = block_peel<NT>(off, adj, n, pp, qq, L, A, R, K0, I0, I1, width, B.block_deg, S);
                width = block_reduce_u32<NT>(width, true, S);
                range = rounds - 1;
                src = R;
            } else {
                // ---- edge scan: thread per vertex below thread_deg arcs
                // (every lane busy on the many small lists), warp per vertex
                // above
                const int64_t thread_deg = B.thread_deg;
                uint32_t lmn = 0xffffffffu, lmx = 0;
                for (uint32_t u = threadIdx.x; u < n; u += NT) {
                    const int64_t s = off[u], e = off[u + 1];
                    const uint32_t lu = L[u];
                    lmn = min(lmn, lu);
                    lmx = max(lmx, lu);
                    if (e - s >= thread_deg) continue;
                    uint32_t c = 0;
                    #pragma unroll 4
                    for (int64_t j = s; j < e; ++j) {
                        const uint32_t w = (uint32_t)adj[j];
                        const uint32_t lw = L[w];
                        c += (lw > lu) || (lw == lu && w > u);
                    }
                    A[u] = c;
                    width = max(width, c);
                }
                for (uint32_t u = warp; u < n; u += NW) {
                    const int64_t s = off[u], e = off[u + 1];
                    if (e - s < thread_deg) continue;
                    const uint32_t lu = L[u];
                    uint32_t c = 0;
                    for (int64_t j = s + lane; j < e; j += 32) {
                        const uint32_t w = (uint32_t)adj[j];
                        const uint32_t lw = L[w];
                        c += (lw > lu) || (lw == lu && w > u);
                    }
                    c = __reduce_add_sync(kFull, c);
                    if (lane == 0) A[u] = c;
                    width = max(width, c);
                }
                width = block_reduce_u32<NT>(width, true, S);
                lmin = block_reduce_u32<NT>(lmn, false, S);
                range = block_reduce_u32<NT>(lmx, true, S) - lmin;
            }
            // ---- sort ids by (key, id): stable LSD passes on key - lmin
            const int bits = range ? 32 - __clz(range) : 0;
            const int np = bits ? (bits + kRadixBits - 1) / kRadixBits : 0;
            const uint32_t *ids;
            const uint32_t *keys;
            if (np == 0) {
                for (uint32_t v = threadIdx.x; v < n; v += NT) { I0[v] = v; K0[v] = 0; }
                __syncthreads();
                ids = I0;
                keys = K0;
            } else {
                const uint32_t *kin = nullptr, *iin = nullptr;
                for (int p = 0; p < np; ++p) {
                    uint32_t *ko = (p & 1) ? K1 : K0, *io = (p & 1) ? I1 : I0;
                    block_radix_pass<NT>(kin, iin, src, lmin, ko, io, n, p * kRadixBits, S);
                    kin = ko;
                    iin = io;
                }
                ids = iin;
                keys = kin;
            }
            // ---- densest suffix: scan of A in order, first maximum
            // kScanK consecutive positions per thread, one block scan per
            // NT * kScanK positions
            Candidate best{0, 0, 0, 0};
            uint64_t carry = 0;
            for (uint32_t c0 = 0; c0 < n; c0 += NT * kScanK) {
                const uint32_t p0 = c0 + threadIdx.x * kScanK;
                uint32_t a[kScanK];
                uint64_t run = 0;
                #pragma unroll
                for (int k = 0; k < kScanK; ++k) {
                    a[k] = p0 + k < n ? A[ids[p0 + k]] : 0u;
                    run += a[k];
                }
                uint64_t tot;
                uint64_t pre = carry + block_excl_sum_u64(run, S.red, &tot);
                #pragma unroll
                for (int k = 0; k < kScanK; ++k) {
                    const uint32_t pos = p0 + k;
                    if (pos < n) {
                        Candidate cd{(int64_t)((uint64_t)m - pre), (int64_t)(n - pos), (int64_t)pos, 0};
                        if (cand_better(cd, best)) best = cd;
                        pre += a[k];
                    }
                }
                carry += tot;
            }
            best = block_best(best, S.cred);
            if (B.trace) {
                if (threadIdx.x == 0) {
                    int64_t *tr = B.trace + ((int64_t)g * B.Tmax + (t - 1)) * 3;
                    tr[0] = best.e;
                    tr[1] = best.v;
                    tr[2] = width;
                }
            }
            const bool improved = best.v > 0 && dens_gt((uint64_t)best.e, (uint64_t)best.v,
                                                        (uint64_t)best_e, (uint64_t)best_v);
            if (improved) {
                best_e = best.e;
                best_v = best.v;
                best_pos = best.pos;
                best_iter = t;
                best_key = keys[best_pos] + lmin;
                best_id = ids[best_pos];
                for (uint32_t v = threadIdx.x; v < n; v += NT) BL[v] = src[v];
            }
            __syncthreads();
            if (!PEEL) {
                for (uint32_t v = threadIdx.x; v < n; v += NT) L[v] += A[v];
                __syncthreads();
            }
        }
        // ---- outputs: loads, best set (ascending ids), summary
        if (B.loads_out)
            for (uint32_t v = threadIdx.x; v < n; v += NT) B.loads_out[vb + v] = (int64_t)L[v];
        uint64_t set_size = 0;
        {
            uint64_t base = 0;
            for (uint32_t c0 = 0; c0 < n; c0 += NT) {
                const uint32_t v = c0 + threadIdx.x;
                bool in = false;
                if (v < n) {
                    if (best_iter == 0) in = true;
                    else {
                        const uint32_t l = BL[v];
                        in = l > best_key || (l == best_key && v >= best_id);
                    }
                }
                uint64_t tot;
                const uint64_t ex = block_excl_sum_u64(in ? 1u : 0u, S.red, &tot);
                if (in && B.sets) B.sets[vb + base + ex] = (int32_t)v;
                base += tot;
            }
            set_size = base;
        }
        if (threadIdx.x == 0) {
            int64_t *o = B.best + 4 * (int64_t)g;
            o[0] = best_e;
            o[1] = best_v;
            o[2] = best_iter;
            o[3] = (int64_t)set_size;
        }
        (void)best_pos;
        __syncthreads();
    }
}

// validation of one graph per block: local ids in range, no self-loop,
// (full) strictly ascending and symmetric lists
__global__ void k_batch_validate(BatchDev B, int full, int32_t *err)
{
    for (int g = blockIdx.x; g < B.G; g += gridDim.x) {
        const int64_t vb = B.vbase[g];
        const int64_t n = B.vbase[g + 1] - vb;
        const int64_t *off = B.off + vb;
        for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
            const int64_t s = off[u], e = off[u + 1];
            if (e < s) { atomicExch(&err[0], 1); continue; }
            for (int64_t j = s; j < e; ++j) {
                const int32_t w = B.adj[j];
                if (w < 0 || w >= n) { atomicExch(&err[1], 1); continue; }
                if (w == (int32_t)u) atomicExch(&err[2], 1);
                if (full) {
                    if (j > s && B.adj[j - 1] >= w) atomicExch(&err[3], 1);
                    int64_t lo = off[w], hi = off[w + 1];
                    bool found = false;
                    while (lo < hi) {
                        const int64_t mid = lo + (hi - lo) / 2;
                        const int32_t x = B.adj[mid];
                        if (x == (int32_t)u) { found = true; break; }
                        if (x < (int32_t)u) lo = mid + 1; else hi = mid;
                    }
                    if (!found) atomicExch(&err[4], 1);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_batch_validate(const BatchDev &B, int full, int32_t *err, cudaStream_t s)
{
    cudaMemsetAsync(err, 0, 8 * sizeof(int32_t), s);
    k_batch_validate<<<(unsigned)imin64(B.G, 152 * 8), 256, 0, s>>>(B, full, err);
    return cudaGetLastError();
}

template <int NT, bool PEEL>
static cudaError_t launch_one(const BatchDev &B, int sm_count, uint32_t *graph_ctr, cudaStream_t s)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_run<NT, PEEL>, NT, 0);
    const int grid = (int)imin64((int64_t)sm_count * (nb > 0 ? nb : 1), B.G);
    k_batch_run<NT, PEEL><<<grid, NT, 0, s>>>(B, graph_ctr);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchDev &B, int variant, int threads, int sm_count, uint32_t *graph_ctr,
                         cudaStream_t s)
{
    cudaMemsetAsync(graph_ctr, 0, sizeof(uint32_t), s);
    const bool peel = variant == DSG_PEELING;
    switch (threads) {
    case 256: return peel ? launch_one<256, true>(B, sm_count, graph_ctr, s) : launch_one<256, false>(B, sm_count, graph_ctr, s);
    case 512: return peel ? launch_one<512, true>(B, sm_count, graph_ctr, s) : launch_one<512, false>(B, sm_count, graph_ctr, s);
    case 1024: return peel ? launch_one<1024, true>(B, sm_count, graph_ctr, s) : launch_one<1024, false>(B, sm_count, graph_ctr, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dsg
