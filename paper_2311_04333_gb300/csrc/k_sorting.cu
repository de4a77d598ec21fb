// k_sorting.cu -- kernels of one PaRSorting++ iteration (arXiv 2311.04333,
// Sec. 3.2 GreedySorting++ and Sec. 3.3 ParallelGreedySorting++ with the
// density and load computation of Alg. 3), plus the once-per-run kernels.
//
// Iteration t, given loads l_t (uint32, by vertex id):
//   plan       : digit layout of (l_t - min l_t) from the min/max reduced by
//                the previous iteration; resets counters.
//   edge scan  : A[u] = #{w in N(u) : (l_t[w], w) > (l_t[u], u)}, the number
//                of neighbours of u later in the (load, id) order.  Because
//                this comparison does not depend on the sorted positions it
//                runs before the sort (Alg. 3's counts, without ranks).
//                Also builds the digit histograms of the sort and the
//                per-digit sums of A used by the fused scan.
//   radix pass : stable LSD onesweep passes over (key = l_t, value = A) with
//                decoupled look-back; pass 0 also writes l_{t+1} = l_t + A
//                (Alg. 3, load update).  The LAST pass does not scatter: it
//                obtains every element's final position i and its prefix sum
//                of A from the look-back, so the suffix (n - i vertices,
//                m - prefix edges) of Alg. 3's suffix step is evaluated in place
//                and reduced to the iteration's first densest suffix.
//   snapshot   : when the iteration beat the best, keeps l_t for the set.
#include <mutex>

#include "common.cuh"

namespace dsg {

// ============================================================ init / plan

__global__ void k_init_ctl(Control *ctl, int64_t m, int64_t n, uint32_t spin_limit, int32_t debug_stall)
{
    ctl->spin_limit = spin_limit;
    ctl->debug_stall = debug_stall;
    ctl->peel_rounds = 0;
    ctl->peel_work = 0;
    ctl->best_e = m;
    ctl->best_v = n;
    ctl->best_pos = 0;
    ctl->best_key = 0;
    ctl->best_iter = 0;
    ctl->improved = 0;
    ctl->err = 0;
    ctl->err_where = 0;
    ctl->mm_min[1] = 0xffffffffu;
    ctl->mm_max[1] = 0;
    ctl->done_ctr = 0;
}

__global__ void k_init_loads(uint32_t *loads, const int64_t *init, int64_t n, Control *ctl)
{
    uint32_t mn = 0xffffffffu, mx = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = init ? (uint32_t)init[v] : 0u;
        loads[v] = l;
        mn = min(mn, l);
        mx = max(mx, l);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ctl->mm_min[1], mn);
        atomicMax(&ctl->mm_max[1], mx);
    }
}

__global__ void k_plan(Control *ctl, int t)
{
    const int tid = threadIdx.x;
    const uint32_t lmin = ctl->mm_min[t & 1], lmax = ctl->mm_max[t & 1];
    const uint32_t range = lmax - lmin;
    const int bits = range ? 32 - __clz(range) : 0;
    const int np = bits ? (bits + kRadixBits - 1) / kRadixBits : 1;
    for (int i = tid; i < kMaxPasses * kBuckets; i += blockDim.x) (&ctl->hist[0][0])[i] = 0;
    for (int i = tid; i < kBuckets; i += blockDim.x) ctl->asum[i] = 0;
    if (tid == 0) {
        ctl->lmin = lmin;
        ctl->lrange = range;
        ctl->npass = np;
        for (int p = 0; p < kMaxPasses; ++p) ctl->shift[p] = p * kRadixBits;
        ctl->item_ctr = 0;
        for (int p = 0; p < kMaxPasses; ++p) ctl->tile_ctr[p] = 0;
        ctl->done_ctr = 0;
        ctl->width = 0;
        ctl->improved = 0;
        ctl->mm_min[(t + 1) & 1] = 0xffffffffu;
        ctl->mm_max[(t + 1) & 1] = 0;
        ctl->epoch += kMaxPasses;
    }
}

cudaError_t launch_init(const GraphDev &g, RunBufs &b, const int64_t *init_dev, int,
                        cudaStream_t s)
{
    k_init_ctl<<<1, 1, 0, s>>>(b.ctl, g.arcs / 2, g.n, b.spin_limit, b.debug_stall);
    int grid = (int)imin64((g.n + 255) / 256, 4096);
    k_init_loads<<<grid, 256, 0, s>>>(b.loads, init_dev, g.n, b.ctl);
    return cudaGetLastError();
}

cudaError_t launch_plan(const GraphDev &, RunBufs &b, int t, cudaStream_t s)
{
    k_plan<<<1, 256, 0, s>>>(b.ctl, t);
    return cudaGetLastError();
}

// ============================================================ edge scan
// Runs on the degree-oriented copy of the graph: every undirected edge
// {u, w} is stored once, at the endpoint u of smaller (degree, id), so the
// edge is compared once: if w is later than u in the (load, id) order the
// edge counts for u (a register count), otherwise for w (an atomic add to
// A[w]; A is zeroed before the kernel).  Targets among the hubs (the
// largest-degree vertices, most of the targets of a power-law graph) read
// their load from a shared-memory copy and add into shared-memory counters
// that are flushed once per block.
// Work units come from an atomic dispenser:
//   units [0, n_items): one chunk of kChunk oriented arcs of a vertex of
//     out-degree > kHeavyDeg;
//   units after that: a light group of 32 consecutive vertices, one per
//     lane.  Out-degrees >= kMidDeg are taken one at a time by the whole
//     warp; the arcs of the smaller ones are packed across the lanes, each
//     arc finding its source lane by a 5-step shuffle binary search.
// The group's lanes also accumulate the digit histograms of (l - lmin).

constexpr int kEsThreads = DSG_ES_THREADS;
constexpr int kEsMinBlocks = 1024 / kEsThreads;
constexpr int kEsUnroll = DSG_ES_UNROLL;        // rounds of 32 arcs in flight per warp
constexpr int64_t kMidDeg = DSG_MID_DEG;
static_assert(kEsUnroll >= 4 && kEsUnroll % 4 == 0, "source map words hold 4 slots");
constexpr int kMapWords = kEsUnroll / 4;        // source-map words per lane

struct EsSmem {
    uint32_t hist[kMaxPasses][kBuckets];
    uint32_t hub_l[kHubs];      // loads of the hubs
    uint32_t hub_c[kHubs];      // counts for the hubs from this block
    uint32_t hub_v[kHubs];      // ids of the hubs
    uint32_t hot_bit;           // kHotBit when the hot tier exists, else 0
    // per warp: source lane (+1) of each of the 256 arcs of a packed batch
    uint8_t srcmap[kEsThreads / 32][32 * kEsUnroll];
};

// per-thread run-length accumulation of the digit count histograms
struct HistAcc {
    uint32_t b[kMaxPasses], c[kMaxPasses];
};

__device__ __forceinline__ void hist_add(HistAcc &h, EsSmem &S, uint32_t key, uint32_t lmin, int np)
{
    const uint32_t x = key - lmin;
    #pragma unroll
    for (int p = 0; p < kMaxPasses; ++p) {
        if (p < np) {
            uint32_t d = (x >> (p * kRadixBits)) & (kBuckets - 1);
            if (d != h.b[p]) {
                if (h.c[p]) atomicAdd(&S.hist[p][h.b[p]], h.c[p]);
                h.b[p] = d;
                h.c[p] = 0;
            }
            h.c[p] += 1;
        }
    }
}

__device__ __forceinline__ void hist_flush(HistAcc &h, EsSmem &S, int np)
{
    #pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
        if (p < np && h.c[p]) atomicAdd(&S.hist[p][h.b[p]], h.c[p]);
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// streamed read of one oriented arc
__device__ __forceinline__ uint32_t ld_arc(const uint32_t *p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// load of an arc target: shared-memory copy for hubs, the L2-resident hot
// copy for the next tier, the load array otherwise
__device__ __forceinline__ uint32_t target_load(uint32_t t, const uint32_t *__restrict__ loads,
                                                const uint32_t *__restrict__ hot_l, const EsSmem &S)
{
    if (t & kHubBit) return S.hub_l[t & ~kHubBit];
    if (t & S.hot_bit) return __ldg(hot_l + (t & kSlotMask));
    return __ldg(loads + t);
}

// compare target t (load lw) with source (lu, u): count for u, or add one
// to the target's count: shared-memory counters for hubs, the dense hot-tier
// counters (folded into A after the scan) for the next tier, A otherwise
__device__ __forceinline__ void settle(uint32_t t, uint32_t lw, uint32_t lu, uint32_t u,
                                       const uint32_t *__restrict__ hot_id, EsSmem &S,
                                       uint32_t *A, uint32_t *hot_c, uint32_t &c)
{
    const bool hub = t & kHubBit;
    const bool hot = !hub && (t & S.hot_bit);
    bool later = lw > lu;
    if (lw == lu) {
        const uint32_t w = hub ? S.hub_v[t & ~kHubBit] : (hot ? __ldg(hot_id + (t & kSlotMask)) : t);
        later = w > u;
    }
    if (later) ++c;
    else if (hub) atomicAdd(&S.hub_c[t & ~kHubBit], 1u);
    else if (hot) atomicAdd(&hot_c[t & kSlotMask], 1u);
    else atomicAdd(&A[t], 1u);
}

// the warp processes oriented arcs [a0, a1) of source (lu, u); returns this
// lane's count for u
__device__ __forceinline__ uint32_t warp_arcs(const uint32_t *__restrict__ oadj,
                                              const uint32_t *__restrict__ loads,
                                              const uint32_t *__restrict__ hot_l,
                                              const uint32_t *__restrict__ hot_id, EsSmem &S,
                                              uint32_t *A, uint32_t *hot_c, int64_t a0, int64_t a1, uint32_t lu,
                                              uint32_t u, int lane, uint64_t pol)
{
    uint32_t c = 0;
    for (int64_t j0 = a0; j0 < a1; j0 += 32 * kEsUnroll) {
        uint32_t t[kEsUnroll], lw[kEsUnroll];
        #pragma unroll
        for (int k = 0; k < kEsUnroll; ++k) {
            const int64_t j = j0 + k * 32 + lane;
            t[k] = j < a1 ? ld_arc(oadj + j, pol) : 0u;
        }
        #pragma unroll
        for (int k = 0; k < kEsUnroll; ++k) {
            const int64_t j = j0 + k * 32 + lane;
            lw[k] = j < a1 ? target_load(t[k], loads, hot_l, S) : 0u;
        }
        #pragma unroll
        for (int k = 0; k < kEsUnroll; ++k) {
            const int64_t j = j0 + k * 32 + lane;
            if (j < a1) settle(t[k], lw[k], lu, u, hot_id, S, A, hot_c, c);
        }
    }
    return c;
}

__global__ void __launch_bounds__(kEsThreads, kEsMinBlocks)
k_edge_scan(const int64_t *__restrict__ ooff, const uint32_t *__restrict__ oadj,
            const uint32_t *__restrict__ hub_id, int64_t n_hub,
            const uint32_t *__restrict__ hot_l, const uint32_t *__restrict__ hot_id,
            const WorkItem *__restrict__ items, int64_t n_items, int64_t n,
            const uint32_t *__restrict__ loads, uint32_t *A, uint32_t *hot_c, Control *ctl, int sorted)
{
    extern __shared__ __align__(16) unsigned char es_smem_raw[];
    EsSmem &S = *reinterpret_cast<EsSmem *>(es_smem_raw);
    if (sorted && ctl->lrange == 0) return;    // k_edge_scan_equal does this iteration
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lmin = ctl->lmin;
    const int np = ctl->npass;
    const uint64_t pol = policy_evict_first();
    const int64_t n_units = n_items + (n + 31) / 32;

    for (int i = tid; i < kMaxPasses * kBuckets; i += kEsThreads) (&S.hist[0][0])[i] = 0;
    if (tid == 0) S.hot_bit = hot_id ? kHotBit : 0u;
    for (int i = tid; i < n_hub; i += kEsThreads) {
        const uint32_t v = hub_id[i];
        S.hub_v[i] = v;
        S.hub_l[i] = loads[v];
        S.hub_c[i] = 0;
    }
    HistAcc h;
    #pragma unroll
    for (int p = 0; p < kMaxPasses; ++p) { h.b[p] = 0; h.c[p] = 0; }
    __syncthreads();

    for (;;) {
        uint32_t unit = 0;
        if (lane == 0) unit = atomicAdd(&ctl->item_ctr, 1u);
        unit = __shfl_sync(kFull, unit, 0);
        if ((int64_t)unit >= n_units) break;

        if ((int64_t)unit < n_items) {
            // ---- one chunk of a vertex of large out-degree
            const WorkItem it = items[unit];
            const uint32_t u = it.u;
            const int64_t a1 = imin64(it.a0 + (int64_t)kChunk, ooff[u + 1]);
            uint32_t c = warp_arcs(oadj, loads, hot_l, hot_id, S, A, hot_c, it.a0, a1, loads[u], u, lane, pol);
            c = __reduce_add_sync(kFull, c);
            if (lane == 0 && c) atomicAdd(&A[u], c);
            continue;
        }

        // ---- light group: vertices 32*g .. 32*g+31
        const int64_t g0 = ((int64_t)unit - n_items) * 32;
        const int64_t uu = g0 + lane;
        const bool valid = uu < n;
        const int64_t s = valid ? ooff[uu] : 0;
        int64_t e = __shfl_down_sync(kFull, s, 1);
        if (lane == 31 || uu + 1 >= n) e = valid ? ooff[uu + 1] : 0;
        const int64_t deg = e - s;
        const bool heavy = deg > kHeavyDeg;
        const bool mid = !heavy && deg >= kMidDeg;
        const uint32_t lu = valid ? loads[uu] : 0u;
        if (valid) hist_add(h, S, lu, lmin, np);
        uint32_t cnt = 0;

        // out-degree kMidDeg..kHeavyDeg: the whole warp, one vertex at a time
        uint32_t mm = __ballot_sync(kFull, mid);
        while (mm) {
            const int l = __ffs(mm) - 1;
            mm &= mm - 1;
            const int64_t vs = __shfl_sync(kFull, s, l), ve = __shfl_sync(kFull, e, l);
            const uint32_t vl = __shfl_sync(kFull, lu, l);
            uint32_t c = warp_arcs(oadj, loads, hot_l, hot_id, S, A, hot_c, vs, ve, vl, (uint32_t)(g0 + l), lane, pol);
            c = __reduce_add_sync(kFull, c);
            if (lane == l) cnt = c;
        }

        // smaller out-degrees: arcs packed across the lanes
        const uint32_t sdeg = (valid && !heavy && !mid) ? (uint32_t)deg : 0u;
        uint32_t incl = sdeg;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const uint32_t start = incl - sdeg;
        if (total) {
            // arc j (packed index) of lane L's vertex is at oadj[sg + j + dofs_L]
            const int64_t sg = __shfl_sync(kFull, s, 0);
            const int32_t dofs = (int32_t)(s - sg) - (int32_t)start;
            uint8_t *map = S.srcmap[tid >> 5];
            uint32_t carry = 0;
            for (uint32_t base = 0; base < total; base += 32 * kEsUnroll) {
                // source map of this batch: mark first slots, then fill forward.
                // Each lane owns kMapWords 32-bit words (4 slots each) of the
                // warp's 32 * kEsUnroll slots.
                uint32_t *mw = reinterpret_cast<uint32_t *>(map) + lane * kMapWords;
                #pragma unroll
                for (int i = 0; i < kMapWords; ++i) mw[i] = 0u;
                __syncwarp();
                if (sdeg && start >= base && start < base + 32 * kEsUnroll)
                    map[start - base] = (uint8_t)(lane + 1);
                __syncwarp();
                uint32_t wv[kMapWords];
                uint32_t lm = 0;
                #pragma unroll
                for (int i = 0; i < kMapWords; ++i) {
                    wv[i] = mw[i];
                    #pragma unroll
                    for (int b = 0; b < 4; ++b) lm = max(lm, (wv[i] >> (8 * b)) & 0xffu);
                }
                uint32_t im = lm;
                #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, im, o);
                    if (lane >= o) im = max(im, y);
                }
                uint32_t cur = __shfl_up_sync(kFull, im, 1);
                cur = max(lane ? cur : 0u, carry);
                #pragma unroll
                for (int i = 0; i < kMapWords; ++i) {
                    uint32_t nw = 0;
                    #pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        cur = max(cur, (wv[i] >> (8 * b)) & 0xffu);
                        nw |= cur << (8 * b);
                    }
                    mw[i] = nw;
                }
                carry = __shfl_sync(kFull, cur, 31);
                __syncwarp();
                uint32_t t[kEsUnroll], lw[kEsUnroll], sl_r[kEsUnroll];
                #pragma unroll
                for (int k = 0; k < kEsUnroll; ++k) {
                    const uint32_t j = base + k * 32 + lane;
                    const uint32_t sl = (uint32_t)map[k * 32 + lane] - 1u;
                    const int32_t dsrc = __shfl_sync(kFull, dofs, sl & 31);
                    sl_r[k] = sl & 31;
                    t[k] = j < total ? ld_arc(oadj + sg + (int64_t)j + dsrc, pol) : 0u;
                }
                #pragma unroll
                for (int k = 0; k < kEsUnroll; ++k) {
                    const uint32_t j = base + k * 32 + lane;
                    lw[k] = j < total ? target_load(t[k], loads, hot_l, S) : 0u;
                }
                #pragma unroll
                for (int k = 0; k < kEsUnroll; ++k) {
                    const uint32_t j = base + k * 32 + lane;
                    const uint32_t l_src = __shfl_sync(kFull, lu, sl_r[k]);
                    uint32_t one = 0;
                    if (j < total) settle(t[k], lw[k], l_src, (uint32_t)(g0 + sl_r[k]), hot_id, S, A, hot_c, one);
                    const uint32_t C = __ballot_sync(kFull, one != 0);
                    const int jb = (int)(base + k * 32);
                    const int lo = max((int)start - jb, 0), hi = min((int)incl - jb, 32);
                    if (hi > lo) {
                        const uint32_t mhi = hi == 32 ? kFull : ((1u << hi) - 1u);
                        cnt += __popc(C & mhi & ~((1u << lo) - 1u));
                    }
                }
                __syncwarp();
            }
        }
        if (valid && cnt) atomicAdd(&A[uu], cnt);
    }

    hist_flush(h, S, np);
    __syncthreads();
    for (int i = tid; i < kBuckets; i += kEsThreads)
        for (int p = 0; p < np; ++p)
            if (S.hist[p][i]) atomicAdd(&ctl->hist[p][i], S.hist[p][i]);
    for (int i = tid; i < n_hub; i += kEsThreads)
        if (S.hub_c[i]) atomicAdd(&A[hub_id[i]], S.hub_c[i]);
}

static int g_es_blocks_per_sm = -1;
static std::once_flag g_es_once;

int edge_scan_sm_count()
{
    std::call_once(g_es_once, [] {
        cudaFuncSetAttribute(k_edge_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EsSmem));
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_edge_scan, kEsThreads, sizeof(EsSmem));
        g_es_blocks_per_sm = nb > 0 ? nb : 1;
    });
    return g_es_blocks_per_sm;
}

// All loads equal (e.g. iteration 1 from zero loads): the order is the id
// order, so A[u] = #{w in N(u) : w > u}, read off u's ascending adjacency
// list by a binary search for u.  Exits unless the loads are all equal.
__global__ void k_edge_scan_equal(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                  int64_t n, uint32_t *A, Control *ctl)
{
    if (ctl->lrange != 0) return;
    uint32_t cnt = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = off[u];
        const int64_t e = off[u + 1];
        int64_t hi = e;
        while (lo < hi) {                    // first position with adj > u
            const int64_t mid = lo + (hi - lo) / 2;
            if (adj[mid] > (int32_t)u) hi = mid; else lo = mid + 1;
        }
        A[u] = (uint32_t)(e - lo);
        ++cnt;
    }
    cnt = __reduce_add_sync(kFull, cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctl->hist[0][0], cnt);   // range 0: one bucket
}

// dense copy of the hot tier's loads for this iteration
// A[hot_id[i]] += hot_c[i] (distinct ids; after the scan), and reset hot_c
__global__ void k_hot_fold(uint32_t *__restrict__ hot_c, const uint32_t *__restrict__ hot_id, int64_t n_hot,
                           uint32_t *A)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_hot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = hot_c[i];
        if (c) {
            A[hot_id[i]] += c;
            hot_c[i] = 0;
        }
    }
}

__global__ void k_hot_refresh(const uint32_t *__restrict__ loads, const uint32_t *__restrict__ hot_id,
                              int64_t n_hot, uint32_t *__restrict__ hot_l)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_hot;
         i += (int64_t)gridDim.x * blockDim.x)
        hot_l[i] = loads[hot_id[i]];
}

cudaError_t launch_edge_scan(const GraphDev &g, RunBufs &b, int grid, cudaStream_t s)
{
    cudaMemsetAsync(b.A, 0, sizeof(uint32_t) * (size_t)g.n, s);
    if (g.n_hot > 0) {
        const int hg = (int)imin64((g.n_hot + 255) / 256, 152 * 8);
        k_hot_refresh<<<hg, 256, 0, s>>>(b.loads, g.hot_id, g.n_hot, b.hot_l);
    }
    if (g.sorted) {
        const int eg = (int)imin64((g.n + 255) / 256, 152 * 16);
        k_edge_scan_equal<<<eg, 256, 0, s>>>(g.off, g.adj, g.n, b.A, b.ctl);
    }
    k_edge_scan<<<grid, kEsThreads, sizeof(EsSmem), s>>>(g.ooff, g.oadj, g.hub_id, g.n_hub, b.hot_l,
                                            g.n_hot > 0 ? g.hot_id : nullptr,
                                            g.items, g.n_items, g.n, b.loads, b.A, b.hot_c, b.ctl, g.sorted);
    if (g.n_hot > 0) {
        const int hg = (int)imin64((g.n_hot + 255) / 256, 152 * 8);
        k_hot_fold<<<hg, 256, 0, s>>>(b.hot_c, g.hot_id, g.n_hot, b.A);
    }
    return cudaGetLastError();
}

// per-digit sums of A for a sort of a single pass (pass 0 accumulates them
// itself when it is not the last pass)
__global__ void k_asum_single_pass(const uint32_t *__restrict__ loads,
                                   const uint32_t *__restrict__ A, int64_t n, Control *ctl)
{
    if (ctl->npass != 1) return;
    __shared__ unsigned long long as[kBuckets];
    const uint32_t lmin = ctl->lmin;
    const int sh = ctl->shift[ctl->npass - 1];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) as[i] = 0;
    __syncthreads();
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const bool ok = v < n;
        const uint32_t bk = ok ? ((loads[v] - lmin) >> sh) & (kBuckets - 1) : kBuckets;
        const uint32_t a = ok ? A[v] : 0u;
        // lanes with the same bucket add together (16-bit halves keep the
        // 32-bit warp sums exact)
        const uint32_t peers = __match_any_sync(kFull, bk);
        const uint32_t lo = __reduce_add_sync(peers, a & 0xffffu);
        const uint32_t hi = __reduce_add_sync(peers, a >> 16);
        if (ok && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
            atomicAdd(&as[bk], (unsigned long long)lo + ((unsigned long long)hi << 16));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
        if (as[i]) atomicAdd(&ctl->asum[i], as[i]);
}

cudaError_t launch_asum_single_pass(const GraphDev &g, RunBufs &b, cudaStream_t s)
{
    const int grid = (int)imin64((g.n + 255) / 256, 152 * 8);
    k_asum_single_pass<<<grid, 256, 0, s>>>(b.loads, b.A, g.n, b.ctl);
    return cudaGetLastError();
}

// ============================================================ radix passes

// one pad word every 32 entries: thread-contiguous and striped accesses
// to the tile are both free of bank conflicts
__device__ __forceinline__ uint32_t pad(uint32_t lp) { return lp + (lp >> 5); }

// shared memory of a pass with IPT items per thread; the per-digit value
// sums and candidates only exist in the last pass
template <int IPT, bool LAST>
struct PassSmem {
    static constexpr int kTile = kPassThreads * IPT;
    static constexpr int kLastB = LAST ? kBuckets : 1;
    uint32_t keys[kTile + kTile / 32];
    uint32_t vals[kTile + kTile / 32];
    alignas(8) uint32_t wcnt[kPassThreads / 32][kBuckets];   // (last pass: chunk offsets after the local sort)
    uint32_t toff[kBuckets + 1];
    uint32_t boff[kBuckets];
    uint32_t gbase[kBuckets];
    unsigned long long aoff[kLastB];
    unsigned long long gsum[kLastB];
    unsigned long long dscan[kLastB];
    unsigned long long dsum[kLastB];       // per-digit sum of the tile's values (last pass)
    unsigned long long asum_acc[kBuckets];
    unsigned long long red[33];
    Candidate cred[LAST ? 32 : 1];
    uint32_t tile;
    uint32_t last_block;
    uint32_t mn[kPassThreads / 32], mx[kPassThreads / 32];
};

#ifndef DSG_PASS_MINBLOCKS
#define DSG_PASS_MINBLOCKS 3
#endif
#ifndef DSG_PASS_MINBLOCKS_SCATTER
#define DSG_PASS_MINBLOCKS_SCATTER 3
#endif
__device__ __forceinline__ unsigned long long status_word(uint32_t epoch, uint64_t flag, uint64_t cnt)
{
    return ((unsigned long long)epoch << 48) | (flag << 46) | (cnt & ((1ull << 46) - 1));
}
// value sums of the last pass carry the epoch in their top 16 bits, so a
// reader that sees a tile's status word before its sum can tell a stale sum
// (sums stay below m < 2^48)
constexpr unsigned long long kSumMask = (1ull << 48) - 1;
__device__ __forceinline__ unsigned long long sum_word(uint32_t epoch, uint64_t sum)
{
    return ((unsigned long long)epoch << 48) | (sum & kSumMask);
}
// tiles whose status words one look-back step loads at once
constexpr int kLookWin = 8;

// One LSD pass (digit k of key - lmin) over (key, value) pairs, stable.
// Each tile of kPassTile elements: load, rank within warps by match.any,
// publish its per-digit counts (and, in the last pass, value sums) at once,
// sort locally in shared memory, then resolve its global offsets by
// decoupled look-back.  Non-last passes scatter; the last pass evaluates the
// suffix starting at every element's final position (Alg. 3, suffix densities).
// Scatter passes and the last pass are separate instantiations (LAST), each
// with its own tile (IPT items per thread) and residency.  The host launches
// the scatter instantiation for passes 0 .. kMaxPasses - 2 (a launch whose
// pass is not a scatter pass returns at once) and the last instantiation
// once, which takes its pass index np - 1 from the plan on the device.
template <int IPT, bool LAST>
__global__ void __launch_bounds__(kPassThreads, LAST ? DSG_PASS_MINBLOCKS : DSG_PASS_MINBLOCKS_SCATTER)
k_radix_pass(PassIo io, uint32_t *loads_next, unsigned long long *status, unsigned long long *status_sum,
             Candidate *cand, int64_t ntiles, int64_t n, int64_t m, Control *ctl, int kk, int t,
             int64_t *trace, int accumulate)
{
    constexpr int kPassIpt = IPT;
    constexpr int kPassTile = kPassThreads * IPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassSmem<IPT, LAST> &S = *reinterpret_cast<PassSmem<IPT, LAST> *>(smem_raw);
    const int np = ctl->npass;
    const int k = LAST ? np - 1 : kk;
    if (LAST ? (k < 0 || k >= kMaxPasses) : k >= np - 1) return;
    // pass k reads (key0, val0) by id when k == 0, else the buffers pass
    // k - 1 wrote; it writes buffer k & 1
    const uint32_t *kin = k == 0 ? io.key0 : (((k - 1) & 1) ? io.keys1 : io.keys0);
    const uint32_t *vin = k == 0 ? io.val0 : (((k - 1) & 1) ? io.vals1 : io.vals0);
    uint32_t *__restrict__ kout = (k & 1) ? io.keys1 : io.keys0;
    uint32_t *__restrict__ vout = (k & 1) ? io.vals1 : io.vals0;
    constexpr bool last = LAST;
    if (last && ((uint64_t)m >> 48)) {      // sums must fit the tagged words (every block returns)
        if (threadIdx.x == 0 && blockIdx.x == 0) set_error(ctl, 3, 400 + k);
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lmin = ctl->lmin;
    const int shift = ctl->shift[k];
    const uint32_t epoch = (uint32_t)(((ctl->epoch + (uint32_t)k) % 65535u) + 1u);

    if (tid == 0) {
        S.tile = atomicAdd(&ctl->tile_ctr[k], 1u);
        S.last_block = 0;
    }
    for (int i = tid; i < (kPassThreads / 32) * kBuckets; i += kPassThreads) (&S.wcnt[0][0])[i] = 0;
    S.asum_acc[tid] = 0;
    __syncthreads();
    const uint32_t tile = S.tile;
    const int64_t tbase = (int64_t)tile * kPassTile;

    // ---- keys: kPassIpt rounds of 32 consecutive items per warp (all loads
    // first; indices inside the warp's segment are 32-bit).  The values are
    // loaded once the keys are ranked, so the ranking loop holds only the
    // keys and their ranks.
    uint32_t key_r[kPassIpt], rk_r[(kPassIpt + 1) / 2];
    const int64_t wbase = tbase + warp * (32 * kPassIpt);
    const int wrem = (int)imax64(0, imin64(n - wbase, (int64_t)(32 * kPassIpt)));   // valid items of the segment
    const uint32_t *kin_w = kin + wbase;
    const uint32_t *vin_w = vin + wbase;
    #pragma unroll
    for (int r = 0; r < kPassIpt; ++r) {
        const int li = r * 32 + lane;
        key_r[r] = li < wrem ? kin_w[li] : 0u;
    }
    // global bucket offsets of this pass's digit (overlaps the loads)
    {
        const uint32_t hcount = ctl->hist[k][tid];
        uint64_t tot;
        S.boff[tid] = (uint32_t)block_excl_sum_u64(hcount, S.red, &tot);
        if (last) S.aoff[tid] = block_excl_sum_u64(ctl->asum[tid], S.red, &tot);
    }

    // ---- warp-level stable ranks (lanes of equal digit); a rank is below
    // 32 * kPassIpt, so two fit one register
    #pragma unroll
    for (int r = 0; r < kPassIpt; ++r) {
        const int li = r * 32 + lane;
        const bool valid = li < wrem;
        const uint32_t d = ((key_r[r] - lmin) >> shift) & (kBuckets - 1);
        // lanes with the same digit (invalid lanes match only themselves)
        uint32_t peers = __match_any_sync(kFull, valid ? d : (uint32_t)kBuckets + lane);
        if (!valid) peers = 0;
        const uint32_t rank = __popc(peers & lanemask_lt());
        const bool leader = valid && (peers >> lane) == 1u;
        uint32_t before = 0;
        if (valid) before = S.wcnt[warp][d];
        __syncwarp();
        if (leader) S.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        const uint32_t wr = before + rank;
        if (r & 1) rk_r[r >> 1] |= wr << 16;
        else rk_r[r >> 1] = wr;
    }
    __syncthreads();

    // ---- per-digit tile counts; publish the count aggregate at once (the
    // last pass publishes its value sums after the local scan below; a
    // reader checks each word's epoch, so the two need no ordering)
    const int d = tid;
    uint32_t tcount = 0;
    #pragma unroll
    for (int w = 0; w < kPassThreads / 32; ++w) {
        const uint32_t c = S.wcnt[w][d];
        S.wcnt[w][d] = tcount;
        tcount += c;
    }
    unsigned long long *st = status + (int64_t)tile * kBuckets + d;
    unsigned long long *ss = status_sum + 2 * ((int64_t)tile * kBuckets + d);
    // (test-only: debug_stall 1 withholds tile 0's words, so that the
    // look-back of tile 1 waits on words nothing sets and gives up)
    const bool withhold = tile == 0 && ctl->debug_stall == 1;
    if (!withhold) st_relaxed(st, status_word(epoch, tile == 0 ? kFlagIncl : kFlagAgg, tcount));
    {
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(tcount, S.red, &tot);
        S.toff[d] = (uint32_t)ex;
        if (d == 0) S.toff[kBuckets] = (uint32_t)tot;
        // per-warp local start of digit d (thread d owns column d)
        #pragma unroll
        for (int w = 0; w < kPassThreads / 32; ++w) S.wcnt[w][d] += (uint32_t)ex;
    }
    __syncthreads();

    // ---- local stable sort of the tile into shared memory: the keys from
    // registers (each item's local position replaces its rank), then the
    // values, loaded now.  The first pass also writes the next loads l + A by
    // id and gathers the statistics of the loaded pairs.
    #pragma unroll
    for (int r = 0; r < kPassIpt; ++r) {
        const int li = r * 32 + lane;
        const uint32_t half = (rk_r[r >> 1] >> ((r & 1) * 16)) & 0xffffu;
        uint32_t lp = 0;
        if (li < wrem) {
            const uint32_t key = key_r[r];
            const uint32_t dd = ((key - lmin) >> shift) & (kBuckets - 1);
            lp = S.wcnt[warp][dd] + half;
            S.keys[pad(lp)] = key;
        }
        if (r & 1) rk_r[r >> 1] = (rk_r[r >> 1] & 0xffffu) | (lp << 16);
        else rk_r[r >> 1] = (rk_r[r >> 1] & 0xffff0000u) | lp;
    }
    uint32_t lmn = 0xffffffffu, lmx = 0, amax = 0, rb = 0;
    unsigned long long rs = 0;
    const bool acc = accumulate && k == 0;
    const int shift_last = ctl->shift[np - 1];
    uint32_t val_r[kPassIpt];
    #pragma unroll
    for (int r = 0; r < kPassIpt; ++r) {
        const int li = r * 32 + lane;
        val_r[r] = li < wrem ? vin_w[li] : 0u;
    }
    #pragma unroll
    for (int r = 0; r < kPassIpt; ++r) {
        const int li = r * 32 + lane;
        if (li < wrem) {
            const uint32_t lp = (rk_r[r >> 1] >> ((r & 1) * 16)) & 0xffffu;
            S.vals[pad(lp)] = val_r[r];
        }
    }
    if (k == 0 && (loads_next || acc)) {
        #pragma unroll
        for (int r = 0; r < kPassIpt; ++r) {
            const int li = r * 32 + lane;
            if (li < wrem) {
                const uint32_t val = val_r[r];
                const uint32_t lp = (rk_r[r >> 1] >> ((r & 1) * 16)) & 0xffffu;
                const uint32_t key = S.keys[pad(lp)];
                if (loads_next) {
                    const uint32_t nl = key + val;
                    loads_next[wbase + li] = nl;
                    lmn = min(lmn, nl);
                    lmx = max(lmx, nl);
                }
                if (acc) {
                    amax = max(amax, val);
                    if (!last) {
                        const uint32_t dl = ((key - lmin) >> shift_last) & (kBuckets - 1);
                        if (dl != rb) {
                            if (rs) atomicAdd(&S.asum_acc[rb], rs);
                            rb = dl;
                            rs = 0;
                        }
                        rs += val;
                    }
                }
            }
        }
    }
    if (acc) {
        if (!last && rs) atomicAdd(&S.asum_acc[rb], rs);
        amax = __reduce_max_sync(kFull, amax);
        if (lane == 0 && amax) atomicMax(&ctl->width, amax);
    }
    if (k == 0 && loads_next) {
        lmn = __reduce_min_sync(kFull, lmn);
        lmx = __reduce_max_sync(kFull, lmx);
        if (lane == 0) { S.mn[warp] = lmn; S.mx[warp] = lmx; }
    }
    __syncthreads();
    const uint32_t tn = S.toff[kBuckets];
    if (acc && !last && S.asum_acc[tid]) atomicAdd(&ctl->asum[tid], S.asum_acc[tid]);
    if (k == 0 && loads_next && tid == 0) {
        uint32_t a = 0xffffffffu, b = 0;
        for (int i = 0; i < kPassThreads / 32; ++i) { a = min(a, S.mn[i]); b = max(b, S.mx[i]); }
        atomicMin(&ctl->mm_min[(t + 1) & 1], a);
        atomicMax(&ctl->mm_max[(t + 1) & 1], b);
    }

    // last pass: exclusive scan of the values over the locally sorted tile;
    // each thread keeps only its chunk's offset (the per-element values are
    // recomputed after the look-back).  dscan[d] = the scan at digit d's
    // first local position toff[d], found from the chunk holding it, so the
    // digit's value sum is dscan[d + 1] - dscan[d].
    uint64_t chunk_ex = 0, tsum = 0;
    if (last) {
        uint64_t run = 0;
        #pragma unroll
        for (int i = 0; i < kPassIpt; ++i) {
            const uint32_t lp = tid * kPassIpt + i;
            run += lp < tn ? S.vals[pad(lp)] : 0u;
        }
        uint64_t tot;
        chunk_ex = block_excl_sum_u64(run, S.red, &tot);
        unsigned long long *cex = reinterpret_cast<unsigned long long *>(&S.wcnt[0][0]);   // free after the local sort
        cex[tid] = chunk_ex;
        __syncthreads();
        {
            const uint32_t p0 = S.toff[d];
            uint64_t P = tot;
            if (p0 < tn) {
                const uint32_t ct = p0 / kPassIpt, ci = p0 - ct * kPassIpt;
                P = cex[ct];
                for (uint32_t j = 0; j < ci; ++j) P += S.vals[pad(ct * kPassIpt + j)];
            }
            S.dscan[d] = P;
        }
        __syncthreads();     // dscan is read by digit below
        tsum = (d + 1 < kBuckets ? (uint64_t)S.dscan[d + 1] : tot) - S.dscan[d];
        if (!withhold) st_relaxed(tile == 0 ? ss + 1 : ss, sum_word(epoch, tsum));
    }
    // ---- decoupled look-back: thread d resolves digit d.  Every status word
    // carries its own count and every sum its own epoch, so the words need no
    // ordering among themselves: each step loads the words (and sums) of
    // kLookWin predecessors at once and consumes them in order up to the
    // first inclusive one, or up to one not yet published (then reloads).
    {
        uint64_t excl = 0, excl_sum = 0;
        bool abort = false;
        if (tile > 0) {
            int64_t j = (int64_t)tile - 1;
            const uint32_t limit = spin_limit_of(ctl->spin_limit);
            uint32_t polls = 0, ns = 8;
            bool done = false;
            while (!done) {
                unsigned long long wv[kLookWin], sv[kLookWin];
                #pragma unroll
                for (int q = 0; q < kLookWin; ++q) {
                    const int64_t jj = j - q;
                    wv[q] = jj >= 0 ? ld_relaxed(status + jj * kBuckets + d) : 0ull;
                }
                if (last) {
                    // the sum slot a word's flag selects: aggregate [0], inclusive [1]
                    #pragma unroll
                    for (int q = 0; q < kLookWin; ++q) {
                        const int64_t jj = j - q;
                        const uint32_t fl = (uint32_t)((wv[q] >> 46) & 3u);
                        sv[q] = jj >= 0 ? ld_relaxed(status_sum + 2 * (jj * kBuckets + d) + (fl == kFlagIncl ? 1 : 0))
                                        : 0ull;
                    }
                }
                int used = 0;
                bool blocked = false;
                #pragma unroll
                for (int q = 0; q < kLookWin; ++q) {
                    if (done || blocked || j - q < 0) continue;
                    const unsigned long long w = wv[q];
                    const uint32_t ep = (uint32_t)(w >> 48);
                    const uint32_t fl = (uint32_t)((w >> 46) & 3u);
                    if (ep != epoch || fl == 0) { blocked = true; continue; }
                    if (fl == kFlagAbort) { abort = true; done = true; continue; }
                    if (last && (uint32_t)(sv[q] >> 48) != epoch) { blocked = true; continue; }
                    excl += w & ((1ull << 46) - 1);
                    if (last) excl_sum += sv[q] & kSumMask;
                    ++used;
                    if (fl == kFlagIncl) done = true;
                }
                j -= used;
                if (done) break;
                if (j < 0) {                 // tile 0 is always inclusive: unreachable
                    abort = true;
                    set_error(ctl, 5, 200 + k);
                    break;
                }
                if (used == 0) {
                    if (++polls > limit) { abort = true; set_error(ctl, 5, 100 + k); break; }
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                }
            }
            if (abort) {
                st_relaxed(st, status_word(epoch, kFlagAbort, 0));
            } else {
                if (last) st_relaxed(ss + 1, sum_word(epoch, excl_sum + tsum));
                st_relaxed(st, status_word(epoch, kFlagIncl, excl + tcount));
            }
        }
        // global position of local position lp of digit d: gbase[d] + lp
        // (modulo 2^32; positions stay below n < 2^31)
        S.gbase[d] = S.boff[d] + (uint32_t)excl - S.toff[d];
        // prefix sum of A before local position lp of digit d: gsum[d] + (the
        // tile's exclusive value scan at lp)
        if (last) S.gsum[d] = S.aoff[d] + excl_sum - S.dscan[d];
        if (abort) S.last_block = 0xdeadu;
    }
    __syncthreads();
    if (S.last_block == 0xdeadu) return;

    if (!last) {
        // scatter the locally sorted tile: consecutive threads write consecutive
        // positions of a bucket
        #pragma unroll 4
        for (int r = 0; r < kPassIpt; ++r) {
            const uint32_t lp = r * kPassThreads + tid;
            if (lp < tn) {
                const uint32_t key = S.keys[pad(lp)];
                const uint32_t dd = ((key - lmin) >> shift) & (kBuckets - 1);
                const uint32_t gp = S.gbase[dd] + lp;
                if (gp < (uint64_t)n) {
                    kout[gp] = key;
                    vout[gp] = S.vals[pad(lp)];
                } else {
                    set_error(ctl, 3, 300 + k);
                }
            }
        }
        return;
    }

    // ---- final pass: evaluate every suffix (Alg. 3, suffix densities) without scattering
    // A thread's elements sit at increasing positions, so on equal density
    // the one it already holds (the earlier, larger suffix) stays.
    Candidate best{0, 0, 0, 0};
    uint64_t run = chunk_ex;
    if ((uint64_t)m >> 32) {
        #pragma unroll
        for (int i = 0; i < kPassIpt; ++i) {
            const uint32_t lp = tid * kPassIpt + i;
            if (lp < tn) {
                const uint32_t key = S.keys[pad(lp)];
                const uint32_t dd = ((key - lmin) >> shift) & (kBuckets - 1);
                const int64_t pos = (int64_t)(uint32_t)(S.gbase[dd] + lp);
                const uint64_t prefix = S.gsum[dd] + run;
                Candidate c{(int64_t)((uint64_t)m - prefix), n - pos, pos, (int64_t)key};
                if (cand_better(c, best)) best = c;
                run += S.vals[pad(lp)];
            }
        }
    } else {
        // m < 2^32 and n < 2^31: every prefix sum and count fits 32 bits (the
        // sums modulo 2^32 are exact), and e * v' < 2^63, so 64-bit cross
        // products compare the densities exactly.  A thread's elements are
        // sorted by digit: its digit advances at the tile's digit starts.
        const uint32_t lp0 = tid * kPassIpt;
        if (lp0 < tn) {
            uint32_t cd = ((S.keys[pad(lp0)] - lmin) >> shift) & (kBuckets - 1);
            uint32_t nb = S.toff[cd + 1];
            uint32_t gb = S.gbase[cd];
            uint32_t gs = (uint32_t)S.gsum[cd] + (uint32_t)chunk_ex;
            const uint32_t m32 = (uint32_t)m, n32 = (uint32_t)n;
            uint32_t be = 0, bv = 0, blp = 0, bpos = 0, run32 = 0;
            #pragma unroll
            for (int i = 0; i < kPassIpt; ++i) {
                const uint32_t lp = lp0 + i;
                if (lp < tn) {
                    if (lp >= nb) {
                        do { ++cd; nb = S.toff[cd + 1]; } while (lp >= nb);
                        gb = S.gbase[cd];
                        gs = (uint32_t)S.gsum[cd] + (uint32_t)chunk_ex;
                    }
                    const uint32_t pos = gb + lp;
                    const uint32_t e = m32 - (gs + run32);
                    const uint32_t v = n32 - pos;
                    if (bv == 0 || (uint64_t)e * bv > (uint64_t)be * v) {
                        be = e; bv = v; bpos = pos; blp = lp;
                    }
                    run32 += S.vals[pad(lp)];
                }
            }
            if (bv) best = Candidate{(int64_t)be, (int64_t)bv, (int64_t)bpos, (int64_t)S.keys[pad(blp)]};
        }
    }
    best = block_best(best, S.cred);
    if (tid == 0) {
        cand[tile] = best;
        __threadfence();
        S.last_block = (atomicAdd(&ctl->done_ctr, 1u) == (uint32_t)(ntiles - 1)) ? 1u : 0u;
    }
    __syncthreads();
    if (!S.last_block) return;
    __threadfence();
    Candidate b2{0, 0, 0, 0};
    for (int64_t i = tid; i < ntiles; i += kPassThreads) {
        Candidate c;
        c.e = __ldcg(&cand[i].e);
        c.v = __ldcg(&cand[i].v);
        c.pos = __ldcg(&cand[i].pos);
        c.key = __ldcg(&cand[i].key);
        if (cand_better(c, b2)) b2 = c;
    }
    b2 = block_best(b2, S.cred);
    if (tid == 0) {
        if (trace) {
            trace[3 * (t - 1) + 0] = b2.e;
            trace[3 * (t - 1) + 1] = b2.v;
            trace[3 * (t - 1) + 2] = (int64_t)ctl->width;
        }
        if (b2.v > 0 && dens_gt((uint64_t)b2.e, (uint64_t)b2.v, (uint64_t)ctl->best_e,
                                (uint64_t)ctl->best_v)) {
            ctl->best_e = b2.e;
            ctl->best_v = b2.v;
            ctl->best_pos = b2.pos;
            ctl->best_key = b2.key;
            ctl->best_iter = t;
            ctl->improved = 1;
        } else {
            ctl->improved = 0;
        }
    }
}

static std::once_flag g_pass_once;
using PassScatter = PassSmem<kPassIptS, false>;
using PassLast = PassSmem<kPassIpt, true>;

void radix_prepare()
{
    std::call_once(g_pass_once, [] {
        cudaFuncSetAttribute(k_radix_pass<kPassIptS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PassScatter));
        cudaFuncSetAttribute(k_radix_pass<kPassIpt, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PassLast));
    });
}

cudaError_t launch_radix_passes(const GraphDev &g, RunBufs &b, int t, cudaStream_t s,
                                const uint32_t *key0, bool update_loads, bool accumulate)
{
    radix_prepare();
    const PassIo io{key0 ? key0 : b.loads, b.A, b.keys[0], b.keys[1], b.vals[0], b.vals[1]};
    uint32_t *ln = update_loads ? b.loads : nullptr;
    for (int k = 0; k < kMaxPasses - 1; ++k)
        k_radix_pass<kPassIptS, false><<<(unsigned)pass_tiles_scatter(g.n), kPassThreads, sizeof(PassScatter), s>>>(
            io, ln, b.status, b.status_sum, b.cand, pass_tiles_scatter(g.n), g.n, g.arcs / 2, b.ctl, k, t, b.trace,
            accumulate ? 1 : 0);
    k_radix_pass<kPassIpt, true><<<(unsigned)pass_tiles_last(g.n), kPassThreads, sizeof(PassLast), s>>>(
        io, ln, b.status, b.status_sum, b.cand, pass_tiles_last(g.n), g.n, g.arcs / 2, b.ctl, -1, t, b.trace,
        accumulate ? 1 : 0);
    return cudaGetLastError();
}

// ============================================================ snapshot

__global__ void k_snapshot(const uint32_t *__restrict__ loads, const uint32_t *__restrict__ A,
                           uint32_t *__restrict__ best_loads, int64_t n, const Control *ctl)
{
    if (!ctl->improved) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        best_loads[v] = loads[v] - A[v];
}

cudaError_t launch_snapshot(const GraphDev &g, RunBufs &b, cudaStream_t s)
{
    int grid = (int)imin64((g.n + 255) / 256, 152 * 8);
    k_snapshot<<<grid, 256, 0, s>>>(b.loads, b.A, b.best_loads, g.n, b.ctl);
    return cudaGetLastError();
}

// ============================================================ best set (once per run)
// S = the last best_v vertices of the (L, id) order of the best iteration,
// L = its starting loads: {v : L(v) > key*} plus the equal-load vertices from
// the (pos* - #{L < key*})-th smallest id on.

constexpr int kBsBlock = 4096;   // ids per block
constexpr int kBsThreads = 256;

__global__ void k_bs_count(const uint32_t *__restrict__ L, int64_t n, Control *ctl, int64_t *cnt_eq)
{
    if (ctl->best_iter == 0) return;
    const uint32_t key = (uint32_t)ctl->best_key;
    const int64_t b0 = (int64_t)blockIdx.x * kBsBlock;
    uint32_t eq = 0, lt = 0;
    for (int i = threadIdx.x; i < kBsBlock; i += kBsThreads) {
        const int64_t v = b0 + i;
        if (v < n) {
            const uint32_t l = L[v];
            eq += l == key;
            lt += l < key;
        }
    }
    eq = __reduce_add_sync(kFull, eq);
    lt = __reduce_add_sync(kFull, lt);
    __shared__ uint32_t se[kBsThreads / 32], sl[kBsThreads / 32];
    if ((threadIdx.x & 31) == 0) { se[threadIdx.x >> 5] = eq; sl[threadIdx.x >> 5] = lt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int i = 0; i < kBsThreads / 32; ++i) { a += se[i]; b += sl[i]; }
        cnt_eq[blockIdx.x] = a;
        atomicAdd((unsigned long long *)&ctl->cnt_less, (unsigned long long)b);
    }
}

// single block: find the block and id of the r-th equal-load vertex
__global__ void k_bs_select(const uint32_t *__restrict__ L, int64_t n, Control *ctl,
                            const int64_t *cnt_eq, int64_t nblk)
{
    if (ctl->best_iter == 0) return;
    __shared__ unsigned long long red[33];
    __shared__ int64_t s_blk, s_base;
    const uint32_t key = (uint32_t)ctl->best_key;
    const int64_t r = ctl->best_pos - ctl->cnt_less;
    if (threadIdx.x == 0) { s_blk = -1; s_base = 0; }
    // scan the block counts in chunks of blockDim.x
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nblk; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const uint64_t x = i < nblk ? (uint64_t)cnt_eq[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(x, red, &tot);
        const int64_t lo = carry + (int64_t)ex, hi = lo + (int64_t)x;
        if (i < nblk && r >= lo && r < hi) { s_blk = i; s_base = lo; }
        carry += (int64_t)tot;
        __syncthreads();
    }
    __syncthreads();
    const int64_t blk = s_blk;
    if (blk < 0) { if (threadIdx.x == 0) set_error(ctl, 3, 200); return; }
    // within block blk: ordered scan over ids
    int64_t seen = s_base;
    const int64_t b0 = blk * kBsBlock;
    for (int c0 = 0; c0 < kBsBlock; c0 += blockDim.x) {
        const int64_t v = b0 + c0 + threadIdx.x;
        const uint64_t x = (v < n && L[v] == key) ? 1 : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(x, red, &tot);
        if (x && seen + (int64_t)ex == r) ctl->thr_id = v;
        seen += (int64_t)tot;
        __syncthreads();
    }
}

__device__ __forceinline__ bool bs_member(uint32_t l, int64_t v, uint32_t key, int64_t thr)
{
    return l > key || (l == key && v >= thr);
}

__global__ void k_bs_flagcount(const uint32_t *__restrict__ L, int64_t n, const Control *ctl,
                               int64_t *cnt)
{
    const bool all = ctl->best_iter == 0;
    const uint32_t key = (uint32_t)ctl->best_key;
    const int64_t thr = ctl->thr_id;
    const int64_t b0 = (int64_t)blockIdx.x * kBsBlock;
    uint32_t c = 0;
    for (int i = threadIdx.x; i < kBsBlock; i += kBsThreads) {
        const int64_t v = b0 + i;
        if (v < n) c += all || bs_member(L[v], v, key, thr);
    }
    c = __reduce_add_sync(kFull, c);
    __shared__ uint32_t s[kBsThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int i = 0; i < kBsThreads / 32; ++i) a += s[i];
        cnt[blockIdx.x] = a;
    }
}

__global__ void k_bs_scan(int64_t *cnt, int64_t nblk, Control *ctl)
{
    __shared__ unsigned long long red[33];
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nblk; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const uint64_t x = i < nblk ? (uint64_t)cnt[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(x, red, &tot);
        if (i < nblk) cnt[i] = carry + (int64_t)ex;
        carry += (int64_t)tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) ctl->set_size = carry;
}

__global__ void k_bs_write(const uint32_t *__restrict__ L, int64_t n, const Control *ctl,
                           const int64_t *offs, int32_t *__restrict__ set)
{
    __shared__ unsigned long long red[33];
    const bool all = ctl->best_iter == 0;
    const uint32_t key = (uint32_t)ctl->best_key;
    const int64_t thr = ctl->thr_id;
    const int64_t b0 = (int64_t)blockIdx.x * kBsBlock;
    int64_t base = offs[blockIdx.x];
    for (int c0 = 0; c0 < kBsBlock; c0 += kBsThreads) {
        const int64_t v = b0 + c0 + threadIdx.x;
        const uint64_t x = (v < n && (all || bs_member(L[v], v, key, thr))) ? 1 : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(x, red, &tot);
        if (x) set[base + (int64_t)ex] = (int32_t)v;
        base += (int64_t)tot;
        __syncthreads();
    }
}

__global__ void k_zero_i64(int64_t *p) { *p = 0; }

cudaError_t launch_best_set(const GraphDev &g, RunBufs &b, int32_t *set_dev, cudaStream_t s,
                            int *launches)
{
    const int64_t nblk = (g.n + kBsBlock - 1) / kBsBlock;
    k_zero_i64<<<1, 1, 0, s>>>(&b.ctl->cnt_less);
    k_bs_count<<<(unsigned)nblk, kBsThreads, 0, s>>>(b.best_loads, g.n, b.ctl, b.blk_a);
    k_bs_select<<<1, 1024, 0, s>>>(b.best_loads, g.n, b.ctl, b.blk_a, nblk);
    k_bs_flagcount<<<(unsigned)nblk, kBsThreads, 0, s>>>(b.best_loads, g.n, b.ctl, b.blk_b);
    k_bs_scan<<<1, 1024, 0, s>>>(b.blk_b, nblk, b.ctl);
    int nl = 5;
    if (set_dev) {
        k_bs_write<<<(unsigned)nblk, kBsThreads, 0, s>>>(b.best_loads, g.n, b.ctl, b.blk_b, set_dev);
        ++nl;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

// ============================================================ outputs

__global__ void k_loads_out(const uint32_t *__restrict__ loads, int64_t *__restrict__ dst, int64_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        dst[v] = (int64_t)loads[v];
}

cudaError_t launch_loads_out(const GraphDev &g, RunBufs &b, int64_t *dst, cudaStream_t s)
{
    int grid = (int)imin64((g.n + 255) / 256, 152 * 8);
    k_loads_out<<<grid, 256, 0, s>>>(b.loads, dst, g.n);
    return cudaGetLastError();
}

}  // namespace dsg
