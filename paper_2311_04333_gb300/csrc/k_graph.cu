// k_graph.cu -- upload-time kernels: CSR validation and the tile schedule
// of the edge scan, plus small reductions used by the host orchestration.
#include <vector>

#include "common.cuh"

namespace dsg {

// ============================================================ validation
// err_flags[0]: offsets not monotone; [1]: neighbour out of range;
// [2]: self-loop; [3]: list not strictly ascending (duplicate);
// [4]: asymmetric edge (full validation only).

__device__ __forceinline__ bool has_arc(const int64_t *off, const int32_t *adj, int32_t w, int32_t u)
{
    int64_t lo = off[w], hi = off[w + 1];
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int32_t x = adj[mid];
        if (x == u) return true;
        if (x < u) lo = mid + 1; else hi = mid;
    }
    return false;
}

// Vertices of degree > kBigDeg are processed by a whole block (the list of
// them is built first), those of at most kSmallDeg arcs by one thread each,
// the others by one warp each.
constexpr int64_t kBigDeg = 4096;
constexpr uint32_t kSmallDeg = 16;      // lists up to this length: a thread per vertex in the orientation

// the same with the arc's target w = adj[j] already loaded
__device__ __forceinline__ void check_arc_w(const int64_t *off, const int32_t *adj, int64_t n,
                                            int64_t u, int64_t s, int64_t j, int32_t w, int full, int32_t *err)
{
    if (w < 0 || w >= n) { atomicExch(&err[1], 1); return; }
    if (w == (int32_t)u) atomicExch(&err[2], 1);
    if (j > s && adj[j - 1] >= w) atomicExch(&err[5], 1);   // not strictly ascending
    if (full) {
        if (j > s && adj[j - 1] >= w) atomicExch(&err[3], 1);
        if (!has_arc(off, adj, w, (int32_t)u)) atomicExch(&err[4], 1);
    }
}

__device__ __forceinline__ void check_arc(const int64_t *off, const int32_t *adj, int64_t n,
                                          int64_t u, int64_t s, int64_t j, int full, int32_t *err)
{
    check_arc_w(off, adj, n, u, s, j, adj[j], full, err);
}

// offsets monotone and inside [0, arcs]: checked before anything reads adj
__global__ void k_validate_offsets(const int64_t *__restrict__ off, int64_t n, int64_t arcs, int32_t *err)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = off[u], e = off[u + 1];
        if (s < 0 || e > arcs || e < s) atomicExch(&err[0], 1);
    }
}

// adjacency checks on their own (warp per vertex), for graphs uploaded
// without the degree-oriented copy that otherwise carries them
__global__ void k_validate_adjacency(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                     int64_t n, int full, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {
        const int64_t s = off[u], e = off[u + 1];
        for (int64_t j = s + lane; j < e; j += 32) check_arc(off, adj, n, u, s, j, full, err);
    }
}

cudaError_t launch_validate_adjacency(const GraphDev &g, int full, int32_t *err_flags, cudaStream_t s)
{
    const int grid = (int)imax64(1, imin64((g.n + 7) / 8, 152 * 16));
    k_validate_adjacency<<<grid, 256, 0, s>>>(g.off, g.adj, g.n, full, err_flags);
    return cudaGetLastError();
}

// clears the flags and checks the offsets; the adjacency checks (the `full`
// ones too) run in the orientation's count pass or launch_validate_adjacency
cudaError_t launch_validate(const GraphDev &g, int, int32_t *err_flags, cudaStream_t s)
{
    cudaMemsetAsync(err_flags, 0, 8 * sizeof(int32_t), s);
    const int grid = (int)imin64((g.n + 255) / 256, 152 * 16);
    k_validate_offsets<<<grid, 256, 0, s>>>(g.off, g.n, g.arcs, err_flags);
    return cudaGetLastError();
}

// ============================================================ heavy-chunk schedule
// Vertices of degree > kHeavyDeg get ceil(deg / kChunk) work items of
// kChunk arcs each; heavy index h (their accumulator slot) follows id order.

constexpr int kSchedBlock = 4096;                 // vertices per block
constexpr int kSchedPer = kSchedBlock / 256;      // vertices per thread

__device__ __forceinline__ void sched_counts(const int64_t *off, int64_t n, int64_t v0,
                                             uint64_t &h, uint64_t &c)
{
    h = 0;
    c = 0;
    for (int i = 0; i < kSchedPer; ++i) {
        const int64_t v = v0 + i;
        if (v >= n) break;
        const int64_t d = off[v + 1] - off[v];
        if (d > kHeavyDeg) {
            h += 1;
            c += (uint64_t)((d + kChunk - 1) / kChunk);
        }
    }
}

__global__ void k_sched_count(const int64_t *__restrict__ off, int64_t n, int64_t *cnt_h,
                              int64_t *cnt_c)
{
    __shared__ unsigned long long red[33];
    uint64_t h, c, th, tc;
    sched_counts(off, n, (int64_t)blockIdx.x * kSchedBlock + threadIdx.x * kSchedPer, h, c);
    block_excl_sum_u64(h, red, &th);
    block_excl_sum_u64(c, red, &tc);
    if (threadIdx.x == 0) {
        cnt_h[blockIdx.x] = (int64_t)th;
        cnt_c[blockIdx.x] = (int64_t)tc;
    }
}

__global__ void k_sched_write(const int64_t *__restrict__ off, int64_t n, const int64_t *hoff,
                              const int64_t *coff, WorkItem *items)
{
    __shared__ unsigned long long red[33];
    const int64_t v0 = (int64_t)blockIdx.x * kSchedBlock + threadIdx.x * kSchedPer;
    uint64_t h, c, th, tc;
    sched_counts(off, n, v0, h, c);
    int64_t hi = hoff[blockIdx.x] + (int64_t)block_excl_sum_u64(h, red, &th);
    int64_t ci = coff[blockIdx.x] + (int64_t)block_excl_sum_u64(c, red, &tc);
    for (int i = 0; i < kSchedPer; ++i) {
        const int64_t v = v0 + i;
        if (v >= n) break;
        const int64_t s = off[v], d = off[v + 1] - s;
        if (d <= kHeavyDeg) continue;
        for (int64_t a = 0; a < d; a += kChunk) {
            WorkItem it;
            it.a0 = s + a;
            it.u = (uint32_t)v;
            it.info = (uint32_t)hi;
            items[ci++] = it;
        }
        ++hi;
    }
}

// exclusive scan of int64 in place, single block, chunked; writes the total
__global__ void k_scan_single(int64_t *x, int64_t count, int64_t *total)
{
    __shared__ unsigned long long red[33];
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < count; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const uint64_t v = i < count ? (uint64_t)x[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_u64(v, red, &tot);
        if (i < count) x[i] = carry + (int64_t)ex;
        carry += (int64_t)tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

int64_t schedule_tmp_count(int64_t n) { return 2 * ((n + kSchedBlock - 1) / kSchedBlock) + 4; }

// tmp must hold schedule_tmp_count(n) int64
cudaError_t build_schedule(GraphDev &g, void *tmp, size_t tmp_bytes, cudaStream_t s,
                           int64_t *n_items_out, int64_t *n_heavy_out, WorkItem **items_out,
                           uint32_t **heavy_mem_out)
{
    const int64_t nblk = (g.n + kSchedBlock - 1) / kSchedBlock;
    if (tmp_bytes < (size_t)schedule_tmp_count(g.n) * sizeof(int64_t)) return cudaErrorInvalidValue;
    int64_t *ch = (int64_t *)tmp, *cc = ch + nblk, *tot = cc + nblk;
    k_sched_count<<<(unsigned)nblk, 256, 0, s>>>(g.off, g.n, ch, cc);
    k_scan_single<<<1, 1024, 0, s>>>(ch, nblk, tot);
    k_scan_single<<<1, 1024, 0, s>>>(cc, nblk, tot + 1);
    int64_t h_tot[2];
    cudaError_t e = cudaMemcpyAsync(h_tot, tot, sizeof(h_tot), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    WorkItem *items = nullptr;
    uint32_t *hm = nullptr;
    if ((e = dev_malloc((void **)&items, sizeof(WorkItem) * (size_t)imax64(h_tot[1], 1), s)) != cudaSuccess)
        return e;
    if ((e = dev_malloc((void **)&hm, sizeof(uint32_t) * 2 * (size_t)imax64(h_tot[0], 1), s)) != cudaSuccess) {
        cudaFreeAsync(items, s);
        return e;
    }
    cudaMemsetAsync(hm, 0, sizeof(uint32_t) * 2 * (size_t)imax64(h_tot[0], 1), s);
    k_sched_write<<<(unsigned)nblk, 256, 0, s>>>(g.off, g.n, ch, cc, items);
    *n_items_out = h_tot[1];
    *n_heavy_out = h_tot[0];
    *items_out = items;
    *heavy_mem_out = hm;
    return cudaGetLastError();
}

// ============================================================ generic scan
// exclusive scan of int64[count] in place (multi-block): per-chunk sums,
// a single-block scan of the chunk sums, then per-chunk rescans with base.
constexpr int kScanChunk = 4096;
constexpr int kScanPer = kScanChunk / 256;

__global__ void k_scan_chunksum(const int64_t *__restrict__ x, int64_t count, int64_t *sums)
{
    __shared__ unsigned long long red[33];
    const int64_t b = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    uint64_t t = 0;
    for (int i = 0; i < kScanPer; ++i)
        if (b + i < count) t += (uint64_t)x[b + i];
    uint64_t tot;
    block_excl_sum_u64(t, red, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = (int64_t)tot;
}

__global__ void k_scan_apply(int64_t *x, int64_t count, const int64_t *base)
{
    __shared__ unsigned long long red[33];
    const int64_t b = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    uint64_t t = 0;
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (b + i < count) ? x[b + i] : 0;
        t += (uint64_t)v[i];
    }
    uint64_t tot;
    int64_t run = base[blockIdx.x] + (int64_t)block_excl_sum_u64(t, red, &tot);
    for (int i = 0; i < kScanPer; ++i) {
        if (b + i < count) x[b + i] = run;
        run += v[i];
    }
}

int64_t scan_tmp_count(int64_t count) { return (count + kScanChunk - 1) / kScanChunk + 2; }

// x[count] -> exclusive prefix sums; *total_dev receives the sum.
cudaError_t scan_exclusive_i64(int64_t *x, int64_t count, int64_t *total_dev, int64_t *tmp,
                               cudaStream_t s)
{
    const int64_t nch = (count + kScanChunk - 1) / kScanChunk;
    if (nch == 0) {
        cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s);
        return cudaGetLastError();
    }
    k_scan_chunksum<<<(unsigned)nch, 256, 0, s>>>(x, count, tmp);
    k_scan_single<<<1, 1024, 0, s>>>(tmp, nch, total_dev);
    k_scan_apply<<<(unsigned)nch, 256, 0, s>>>(x, count, tmp);
    return cudaGetLastError();
}

// x[0, count) += *base, and then (second kernel) *base += *add: the running
// base of scans taken range by range
__global__ void k_add_base(int64_t *x, int64_t count, const int64_t *base)
{
    const int64_t b = *base;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += b;
}

__global__ void k_advance(int64_t *base, const int64_t *add, int64_t *copy_to)
{
    *base += *add;
    if (copy_to) *copy_to = *base;
}

// ============================================================ degree orientation
// Each undirected edge {u, w} is stored once, at the endpoint with the
// smaller (degree, id); the other endpoint is the arc's target.  Targets
// among the hubs (the at most kHubs vertices of largest degree, chosen by a
// degree threshold) are encoded as kHubBit | hub slot, slots in id order.

__global__ void k_count_ge(const int64_t *__restrict__ off, int64_t n, int64_t D,
                           unsigned long long *cnt)
{
    unsigned long long c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        c += (off[v + 1] - off[v]) >= D;
    c = __reduce_add_sync(kFull, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

__global__ void k_hub_flags(const int64_t *__restrict__ off, int64_t n, int64_t D, int64_t *flag)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = (off[v + 1] - off[v]) >= D;
}

// flag[] holds exclusive slot offsets now; hubs are the vertices whose degree
// passes the threshold
__global__ void k_hub_slots(const int64_t *__restrict__ off, int64_t n, int64_t D,
                            const int64_t *slot_pre, int32_t *slot_of, uint32_t *hub_id)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const bool hub = (off[v + 1] - off[v]) >= D;
        slot_of[v] = hub ? (int32_t)slot_pre[v] : -1;
        if (hub) hub_id[slot_pre[v]] = (uint32_t)v;
    }
}

__device__ __forceinline__ bool oriented_keep(uint32_t du, uint32_t u, uint32_t dw, uint32_t w)
{
    return dw > du || (dw == du && w > u);
}

// one-byte degree class, non-decreasing in the degree: the degree itself
// below 128, then four classes per doubling (the leading bit and the two
// after it), at most 223 for degrees below 2^31.  Different classes order
// two degrees; equal classes below 128 mean equal degrees.
__host__ __device__ __forceinline__ uint32_t deg_class(uint32_t d)
{
    if (d < 128) return d;
    int b = 31;
    while (!((d >> b) & 1u)) --b;
    return 128u + (uint32_t)(b - 7) * 4u + ((d >> (b - 2)) & 3u);
}

// keep rule of oriented_keep, decided by the targets' degree classes (one
// byte per vertex, which stays in L2), the exact degree read only when the
// classes tie above 128
__device__ __forceinline__ bool keep_by_class(uint32_t du, uint32_t cu, uint32_t u, uint32_t w,
                                              const uint8_t *__restrict__ cls, const uint32_t *__restrict__ deg32)
{
    const uint32_t cw = cls[w];
    if (cw != cu) return cw > cu;
    if (cu < 128) return w > u;
    return oriented_keep(du, u, deg32[w], w);
}

// deg32[v], its class cls[v] and the encoded arc target enc[v] (hub slot,
// hot slot or id)
__global__ void k_deg_enc(const int64_t *__restrict__ off, int64_t n, const int32_t *__restrict__ hub_of,
                          const int32_t *__restrict__ hot_of, uint32_t *deg32, uint8_t *cls, uint32_t *enc)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        deg32[v] = (uint32_t)(off[v + 1] - off[v]);
        cls[v] = (uint8_t)deg_class(deg32[v]);
        const int32_t hs = hub_of[v];
        const int32_t ts = hot_of ? hot_of[v] : -1;
        enc[v] = hs >= 0 ? (kHubBit | (uint32_t)hs) : (ts >= 0 ? (kHotBit | (uint32_t)ts) : (uint32_t)v);
    }
}

// keep bits of the arcs: bit j of the bitmap is set when arc j (position in
// the symmetric adjacency) stays in the oriented copy.  A warp's 32 arcs
// starting at j0 span at most two bitmap words; neighbouring lists share
// words, hence the atomics.
__device__ __forceinline__ void set_keep_bits(uint32_t *bits, int64_t j0, uint32_t m, int lane)
{
    if (!m) return;
    const int64_t wi = j0 >> 5;
    const int sh = (int)(j0 & 31);
    if (lane == 0) atomicOr(&bits[wi], m << sh);
    if (lane == 1 && sh && (m >> (32 - sh))) atomicOr(&bits[wi + 1], m >> (32 - sh));
}

__device__ __forceinline__ bool keep_bit(const uint32_t *__restrict__ bits, int64_t j)
{
    return (bits[j >> 5] >> (j & 31)) & 1u;
}

// validation of the adjacency (ids, self-loops, order, symmetry) fused with
// the oriented out-degree and the keep bits: warp per vertex of degree <= kBigDeg
__global__ void k_orient_count(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                               int64_t n, int64_t u0, int64_t u1, const uint32_t *__restrict__ deg32,
                               const uint8_t *__restrict__ cls, int full, int32_t *err, int64_t *ocnt,
                               uint32_t *bits)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // lists of at most kSmallDeg arcs: one thread per vertex (a warp per
    // vertex would leave most lanes idle on them)
    for (int64_t u = u0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < u1;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = off[u], e = off[u + 1];
        const uint32_t du = (uint32_t)(e - s);
        if (du > kSmallDeg) continue;
        const uint32_t cu = deg_class(du);
        uint32_t mask = 0;
        int32_t prev = 0;
        for (uint32_t k = 0; k < du; ++k) {
            const int32_t w = __ldcs(adj + s + k);
            if (w < 0 || w >= n) {
                atomicExch(&err[1], 1);
                continue;
            }
            if (w == (int32_t)u) atomicExch(&err[2], 1);
            if (k > 0 && prev >= w) {
                atomicExch(&err[5], 1);                     // not strictly ascending
                if (full) atomicExch(&err[3], 1);
            }
            if (full && !has_arc(off, adj, w, (int32_t)u)) atomicExch(&err[4], 1);
            prev = w;
            if (keep_by_class(du, cu, (uint32_t)u, (uint32_t)w, cls, deg32)) mask |= 1u << k;
        }
        if (mask) {
            const int sh = (int)(s & 31);
            atomicOr(&bits[s >> 5], mask << sh);
            if (sh && (mask >> (32 - sh))) atomicOr(&bits[(s >> 5) + 1], mask >> (32 - sh));
        }
        ocnt[u] = __popc(mask);
    }
    for (int64_t u = u0 + wid; u < u1; u += nw) {
        const int64_t s = off[u], e = off[u + 1];
        const uint32_t du = (uint32_t)(e - s);
        if (du <= kSmallDeg || du > kBigDeg) continue;     // the loop above; k_orient_count_big
        const uint32_t cu = deg_class(du);
        uint32_t c = 0;
        for (int64_t j0 = s; j0 < e; j0 += 32) {
            const int64_t j = j0 + lane;
            bool keep = false;
            if (j < e) {
                const int32_t w = __ldcs(adj + j);         // streamed: the classes stay in L2
                check_arc_w(off, adj, n, u, s, j, w, full, err);
                if (w >= 0 && w < n) keep = keep_by_class(du, cu, (uint32_t)u, (uint32_t)w, cls, deg32);
            }
            const uint32_t m = __ballot_sync(kFull, keep);
            c += __popc(m);
            set_keep_bits(bits, j0, m, lane);
        }
        if (lane == 0) ocnt[u] = c;
    }
}

// the same, one block per vertex of degree > kBigDeg
__global__ void k_orient_count_big(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                   int64_t n, int64_t u0, int64_t u1, const uint32_t *__restrict__ deg32,
                                   const uint8_t *__restrict__ cls, const uint32_t *__restrict__ big,
                                   int64_t n_big, int full,
                                   int32_t *err, int64_t *ocnt, uint32_t *bits)
{
    __shared__ uint32_t red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < n_big; b += gridDim.x) {
        const int64_t u = big[b];
        if (u < u0 || u >= u1) continue;                    // the block's uniform choice
        const int64_t s = off[u], e = off[u + 1];
        const uint32_t du = (uint32_t)(e - s), cu = deg_class(du);
        uint32_t c = 0;
        for (int64_t j0 = s; j0 < e; j0 += blockDim.x) {
            const int64_t j = j0 + threadIdx.x;
            bool keep = false;
            if (j < e) {
                const int32_t w = __ldcs(adj + j);         // streamed: the classes stay in L2
                check_arc_w(off, adj, n, u, s, j, w, full, err);
                if (w >= 0 && w < n) keep = keep_by_class(du, cu, (uint32_t)u, (uint32_t)w, cls, deg32);
            }
            const uint32_t m = __ballot_sync(kFull, keep);
            c += __popc(m);
            set_keep_bits(bits, j0 + 32 * warp, m, lane);
        }
        __syncthreads();
        if (lane == 0) red[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            ocnt[u] = t;
        }
    }
}

// warp per vertex of degree <= kBigDeg in [u0, u1): the kept targets in list
// order (the keep bits spare a second gather of the targets' degrees).  A
// position at or beyond cap (oadj's size) is not written; it sets *ovf.
__global__ void k_orient_fill(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                              int64_t u0, int64_t u1, const int64_t *__restrict__ ooff,
                              const uint32_t *__restrict__ bits, const uint32_t *__restrict__ enc,
                              uint32_t *oadj, int64_t cap, int32_t *ovf)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = u0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < u1;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = off[u], e = off[u + 1];
        if ((uint64_t)(e - s) > kSmallDeg) continue;
        int64_t o = ooff[u];
        for (int64_t j = s; j < e; ++j) {
            if (!keep_bit(bits, j)) continue;
            if (o < cap) oadj[o] = enc[__ldcs(adj + j)];
            else atomicExch(ovf, 1);
            ++o;
        }
    }
    for (int64_t u = u0 + wid; u < u1; u += nw) {
        const int64_t s = off[u], e = off[u + 1];
        if ((uint64_t)(e - s) <= kSmallDeg || (uint64_t)(e - s) > kBigDeg) continue;
        int64_t o = ooff[u];
        for (int64_t j0 = s; j0 < e; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool keep = j < e && keep_bit(bits, j);
            const uint32_t m = __ballot_sync(kFull, keep);
            if (keep) {
                const int64_t pos = o + __popc(m & lanemask_lt());
                if (pos < cap) oadj[pos] = enc[adj[j]];
                else atomicExch(ovf, 1);
            }
            o += __popc(m);
        }
    }
}

// one block per vertex of degree > kBigDeg
__global__ void k_orient_fill_big(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                  int64_t u0, int64_t u1, const int64_t *__restrict__ ooff,
                                  const uint32_t *__restrict__ bits, const uint32_t *__restrict__ enc,
                                  const uint32_t *__restrict__ big, int64_t n_big, uint32_t *oadj, int64_t cap,
                                  int32_t *ovf)
{
    __shared__ uint32_t wc[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t b = blockIdx.x; b < n_big; b += gridDim.x) {
        const int64_t u = big[b];
        if (u < u0 || u >= u1) continue;                    // the block's uniform choice
        const int64_t s = off[u], e = off[u + 1];
        int64_t o = ooff[u];
        for (int64_t j0 = s; j0 < e; j0 += blockDim.x) {
            const int64_t j = j0 + threadIdx.x;
            const bool keep = j < e && keep_bit(bits, j);
            const uint32_t m = __ballot_sync(kFull, keep);
            __syncthreads();
            if (lane == 0) wc[warp] = __popc(m);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t t = 0;
                for (int i = 0; i < nwarp; ++i) { const uint32_t c = wc[i]; wc[i] = t; t += c; }
                wc[32] = t;
            }
            __syncthreads();
            if (keep) {
                const int64_t pos = o + wc[warp] + __popc(m & lanemask_lt());
                if (pos < cap) oadj[pos] = enc[adj[j]];
                else atomicExch(ovf, 1);
            }
            o += wc[32];
        }
    }
}

// exact degree histogram up to kDegHist - 1; larger degrees share the last
// bucket (warp-aggregated shared-memory counts for small degrees)
constexpr int kDegHist = 1 << 16;
constexpr int kDegSmem = 2048;
__global__ void k_degree_hist(const int64_t *__restrict__ off, int64_t n, unsigned int *hist)
{
    __shared__ unsigned int sh[kDegSmem];
    for (int i = threadIdx.x; i < kDegSmem; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        const int d = v < n ? (int)imin64(off[v + 1] - off[v], kDegHist - 1) : -1;
        const unsigned peers = __match_any_sync(kFull, d);
        if (d >= 0 && (peers & lanemask_lt()) == 0) {
            if (d < kDegSmem) atomicAdd(&sh[d], (unsigned)__popc(peers));
            else atomicAdd(&hist[d], (unsigned)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kDegSmem; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// smallest D >= 2 with #{deg >= D} <= cap (count(deg >= max_degree + 1) = 0),
// from the degree histogram when the answer lies below its last bucket,
// otherwise by bisection with counting passes
static cudaError_t degree_threshold(const GraphDev &g, int64_t cap, const std::vector<unsigned int> &hist,
                                    unsigned long long *cnt, int grid, cudaStream_t s, int64_t *D_out)
{
    if (g.n <= cap) {                           // every vertex of degree >= 2 fits
        *D_out = 2;
        return cudaSuccess;
    }
    if ((int64_t)hist[kDegHist - 1] <= cap) {
        int64_t above = hist[kDegHist - 1];     // #{deg >= D} for D = kDegHist - 1
        int64_t D = kDegHist - 1;
        while (D > 2 && above + (int64_t)hist[D - 1] <= cap) above += hist[--D];
        *D_out = D;
        return cudaSuccess;
    }
    int64_t lo = kDegHist - 1, hi = g.max_degree + 1;
    cudaError_t e;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        unsigned long long h = 0;
        cudaMemsetAsync(cnt, 0, 8, s);
        k_count_ge<<<grid, 256, 0, s>>>(g.off, g.n, mid, cnt);
        cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if ((int64_t)h <= cap) hi = mid; else lo = mid + 1;
    }
    *D_out = lo;
    return cudaSuccess;
}

// Builds ooff, oadj, hub_id and hot_id (allocated here, stream-ordered).
cudaError_t build_orientation(GraphDev &g, cudaStream_t s, int full, int32_t *err, int *sorted_out,
                              int64_t **ooff_out, uint32_t **oadj_out, uint32_t **hub_out,
                              int64_t *n_hub_out, uint32_t **hot_out, int64_t *n_hot_out,
                              const UploadChunks *chunks, int *launches)
{
    const int64_t n = g.n;
    cudaError_t e;
    int nl = 0;
    const int grid = (int)imin64((n + 255) / 256, 152 * 16);
    DevAllocs A(s);
    // hub threshold: the smallest D >= 2 with #{deg >= D} <= kHubs
    unsigned long long *cnt = nullptr;
    int64_t *tmp = nullptr, *flag = nullptr;
    int32_t *slot_of = nullptr, *slot_of_scratch = nullptr;
    const int64_t ntmp = scan_tmp_count(n + 1);
    if ((e = A.get(&cnt, 8)) != cudaSuccess) return e;
    if ((e = A.get(&tmp, 8 * (size_t)(ntmp + 4))) != cudaSuccess) return e;
    if ((e = A.get(&flag, 8 * (size_t)(n + 1))) != cudaSuccess) return e;
    if ((e = A.get(&slot_of, 4 * (size_t)n)) != cudaSuccess) return e;
    if ((e = A.get(&slot_of_scratch, 4 * (size_t)n)) != cudaSuccess) return e;
    std::vector<unsigned int> dh(kDegHist, 0);
    {
        unsigned int *hd = nullptr;
        if ((e = A.get(&hd, 4 * (size_t)kDegHist)) != cudaSuccess) return e;
        cudaMemsetAsync(hd, 0, 4 * (size_t)kDegHist, s);
        k_degree_hist<<<grid, 256, 0, s>>>(g.off, n, hd);
        cudaMemcpyAsync(dh.data(), hd, 4 * (size_t)kDegHist, cudaMemcpyDeviceToHost, s);
        A.release(hd);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    int64_t D = 0;
    if ((e = degree_threshold(g, kHubs, dh, cnt, grid, s, &D)) != cudaSuccess) return e;
    k_hub_flags<<<grid, 256, 0, s>>>(g.off, n, D, flag);
    int64_t *total = tmp + ntmp;
    if ((e = scan_exclusive_i64(flag, n, total, tmp, s)) != cudaSuccess) return e;
    int64_t n_hub = 0;
    cudaMemcpyAsync(&n_hub, total, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    uint32_t *hub = nullptr;
    if ((e = A.get(&hub, 4 * (size_t)imax64(n_hub, 1))) != cudaSuccess) return e;
    k_hub_slots<<<grid, 256, 0, s>>>(g.off, n, D, flag, slot_of, hub);
    // hot tier (only when plain ids stay below kHotBit)
    int32_t *hot_of = nullptr;
    uint32_t *hot = nullptr;
    int64_t n_hot = 0;
    if (n < (int64_t)kHotBit && kHot > 0) {
        int64_t Dh = 0;
        if ((e = degree_threshold(g, kHot, dh, cnt, grid, s, &Dh)) != cudaSuccess) return e;
        if ((e = A.get(&hot_of, 4 * (size_t)n)) != cudaSuccess) return e;
        k_hub_flags<<<grid, 256, 0, s>>>(g.off, n, Dh, flag);
        if ((e = scan_exclusive_i64(flag, n, total, tmp, s)) != cudaSuccess) return e;
        cudaMemcpyAsync(&n_hot, total, 8, cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if ((e = A.get(&hot, 4 * (size_t)imax64(n_hot, 1))) != cudaSuccess) return e;
        k_hub_slots<<<grid, 256, 0, s>>>(g.off, n, Dh, flag, hot_of, hot);
    }
    // 32-bit degrees and encoded targets; list of vertices of degree > kBigDeg
    uint32_t *deg32 = nullptr, *enc = nullptr, *big = nullptr;
    if ((e = A.get(&deg32, 4 * (size_t)n)) != cudaSuccess) return e;
    if ((e = A.get(&enc, 4 * (size_t)n)) != cudaSuccess) return e;
    uint8_t *cls = nullptr;
    if ((e = A.get(&cls, (size_t)n)) != cudaSuccess) return e;
    k_deg_enc<<<grid, 256, 0, s>>>(g.off, n, slot_of, hot_of, deg32, cls, enc);
    k_hub_flags<<<grid, 256, 0, s>>>(g.off, n, kBigDeg + 1, flag);
    if ((e = scan_exclusive_i64(flag, n, total, tmp, s)) != cudaSuccess) return e;
    int64_t n_big = 0;
    cudaMemcpyAsync(&n_big, total, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if ((e = A.get(&big, 4 * (size_t)imax64(n_big, 1))) != cudaSuccess) return e;
    k_hub_slots<<<grid, 256, 0, s>>>(g.off, n, kBigDeg + 1, flag, slot_of_scratch, big);
    // keep bits of the arcs, set by the count pass and read by the fill pass
    uint32_t *bits = nullptr;
    const size_t nbits_words = (size_t)((g.arcs + 31) / 32) + 1;
    if ((e = A.get(&bits, 4 * nbits_words)) != cudaSuccess) return e;
    cudaMemsetAsync(bits, 0, 4 * nbits_words, s);
    // validation fused with the oriented out-degrees
    const int wgrid = (int)imin64((n * 32 + 255) / 256, 152 * 32);
    const int bgrid = (int)imin64(imax64(n_big, 1), 152 * 2);
    const int nch = chunks ? chunks->k : 0;
    int64_t *run = tmp + ntmp + 1;                                  // running base of the chunk scans
    int32_t *ovf = reinterpret_cast<int32_t *>(tmp + ntmp + 2);     // a fill position beyond oadj's size
    int64_t oarcs = 0;
    uint32_t *oadj = nullptr;
    bool pipelined = false;
    const int64_t cap = g.arcs / 2;
    if (nch > 0 && !full) {
        // a host upload in chunks: as soon as a chunk lands, its vertices are
        // counted, their oriented offsets scanned onto the running base and
        // their kept arcs filled, while the later chunks are still copied.
        // oadj gets m entries, exactly the oriented arcs of a symmetric graph;
        // one that needs more (asymmetric input, accepted without
        // DSG_VALIDATE) is counted and filled again below at its own size
        if ((e = A.get(&oadj, 4 * (size_t)imax64(cap, 1))) != cudaSuccess) return e;
        cudaMemsetAsync(run, 0, 16, s);                             // run and ovf
        pipelined = true;
        for (int i = 0; i < nch; ++i) {
            if ((e = cudaStreamWaitEvent(s, chunks->ev[i], 0)) != cudaSuccess) return e;
            const int64_t v0 = chunks->v[i], v1 = chunks->v[i + 1];
            if (v1 <= v0) continue;
            const int cgrid = (int)imin64(((v1 - v0) * 32 + 255) / 256, 152 * 32);
            const int agrid = (int)imin64((v1 - v0 + 255) / 256, 152 * 8);
            k_orient_count<<<cgrid, 256, 0, s>>>(g.off, g.adj, n, v0, v1, deg32, cls, full, err, flag, bits);
            if (n_big)
                k_orient_count_big<<<bgrid, 1024, 0, s>>>(g.off, g.adj, n, v0, v1, deg32, cls, big, n_big, full, err, flag,
                                                          bits);
            if ((e = scan_exclusive_i64(flag + v0, v1 - v0, total, tmp, s)) != cudaSuccess) return e;
            k_add_base<<<agrid, 256, 0, s>>>(flag + v0, v1 - v0, run);
            k_advance<<<1, 1, 0, s>>>(run, total, flag + n);
            k_orient_fill<<<cgrid, 256, 0, s>>>(g.off, g.adj, v0, v1, flag, bits, enc, oadj, cap, ovf);
            if (n_big)
                k_orient_fill_big<<<bgrid, 1024, 0, s>>>(g.off, g.adj, v0, v1, flag, bits, enc, big, n_big, oadj, cap,
                                                         ovf);
            nl += 8 + (n_big ? 2 : 0);
        }
    } else {
        for (int i = 0; i < nch; ++i)
            if ((e = cudaStreamWaitEvent(s, chunks->ev[i], 0)) != cudaSuccess) return e;
        k_orient_count<<<wgrid, 256, 0, s>>>(g.off, g.adj, n, 0, n, deg32, cls, full, err, flag, bits);
        ++nl;
        if (n_big)
            k_orient_count_big<<<bgrid, 1024, 0, s>>>(g.off, g.adj, n, 0, n, deg32, cls, big, n_big, full, err, flag, bits);
    }
    int32_t h_err[8];
    int32_t h_ovf = 0;
    cudaMemcpyAsync(h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, s);
    if (pipelined) {
        cudaMemcpyAsync(&oarcs, run, 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&h_ovf, ovf, 4, cudaMemcpyDeviceToHost, s);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    bool bad = false;
    for (int i = 0; i < 5; ++i) bad |= h_err[i] != 0;
    *sorted_out = h_err[5] ? 0 : 1;
    if (pipelined && (bad || h_ovf || oarcs > cap)) {
        A.release(oadj);
        oadj = nullptr;
        pipelined = false;
        if (!bad) {
            // more oriented arcs than m: the scans replaced the counts, so
            // count again (the keep bits are set again to the same values)
            k_orient_count<<<wgrid, 256, 0, s>>>(g.off, g.adj, n, 0, n, deg32, cls, full, err, flag, bits);
            if (n_big)
                k_orient_count_big<<<bgrid, 1024, 0, s>>>(g.off, g.adj, n, 0, n, deg32, cls, big, n_big, full, err, flag,
                                                          bits);
            nl += 1 + (n_big ? 1 : 0);
        }
    }
    if (!bad && !pipelined) {
        cudaMemsetAsync(flag + n, 0, 8, s);
        if ((e = scan_exclusive_i64(flag, n + 1, total, tmp, s)) != cudaSuccess) return e;
        cudaMemcpyAsync(&oarcs, total, 8, cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if ((e = A.get(&oadj, 4 * (size_t)imax64(oarcs, 1))) != cudaSuccess) return e;
        k_orient_fill<<<wgrid, 256, 0, s>>>(g.off, g.adj, 0, n, flag, bits, enc, oadj, oarcs, ovf);
        if (n_big)
            k_orient_fill_big<<<bgrid, 1024, 0, s>>>(g.off, g.adj, 0, n, flag, bits, enc, big, n_big, oadj, oarcs, ovf);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the outputs go to the caller; A frees the rest (stream-ordered)
    A.keep(flag);
    A.keep(oadj);
    A.keep(hub);
    A.keep(hot);
    *ooff_out = flag;         // n + 1 exclusive prefix sums = oriented offsets
    *oadj_out = oadj;
    *hub_out = hub;
    *n_hub_out = n_hub;
    *hot_out = hot;
    *n_hot_out = n_hot;
    if (launches) *launches = nl;
    return cudaSuccess;
}

// ============================================================ reductions

__global__ void k_max_i64(const int64_t *__restrict__ src, int64_t n, unsigned long long *dst, int *neg)
{
    unsigned long long mx = 0;
    int ng = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = src[i];
        if (x < 0) ng = 1; else mx = max(mx, (unsigned long long)x);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(dst, mx);
        if (ng) atomicExch(neg, 1);
    }
}

cudaError_t launch_max_u64_of_i64(const int64_t *src, int64_t n, unsigned long long *dst,
                                  int *neg_flag, cudaStream_t s)
{
    int grid = (int)imin64((n + 255) / 256, 152 * 8);
    if (grid < 1) grid = 1;
    k_max_i64<<<grid, 256, 0, s>>>(src, n, dst, neg_flag);
    return cudaGetLastError();
}

__global__ void k_degree_max(const int64_t *__restrict__ off, int64_t n, unsigned long long *dst)
{
    unsigned long long mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)(off[i + 1] - off[i]));
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, mx);
}

cudaError_t launch_degree_max(const int64_t *off, int64_t n, unsigned long long *dst, cudaStream_t s)
{
    int grid = (int)imin64((n + 255) / 256, 152 * 8);
    if (grid < 1) grid = 1;
    k_degree_max<<<grid, 256, 0, s>>>(off, n, dst);
    return cudaGetLastError();
}

}  // namespace dsg

namespace dsg {

// ---- host-to-device copy by the SMs -------------------------------------
// On this system the copy engines' host-to-device rate drops well below the
// link's (measured 46-212 GB/s from one copy to the next) while SM loads
// from pinned host memory hold it (211 GB/s).  The kernel copies
// [src, src + bytes) to dst: 16-byte accesses when both addresses share
// their alignment mod 16 (the unaligned head and tail in 4-byte words),
// 4-byte accesses otherwise.  Sizes and addresses are multiples of 4.
__global__ void k_copy_words(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, size_t words)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += stride) dst[i] = src[i];
}

__global__ void k_copy_vec(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}

cudaError_t launch_copy_h2d(const void *src_dev_view, void *dst, size_t bytes, int sm_count, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    if ((bytes & 3) || ((uintptr_t)src_dev_view & 3) || ((uintptr_t)dst & 3)) return cudaErrorInvalidValue;
    // a quarter of the SMs already holds the link's rate (19 blocks of 512
    // threads: 210 GB/s); the other SMs stay free for the kernels that
    // orient the graph as its chunks land, which slowed down by about 1.7x
    // when every SM also ran a copy block (R-MAT 27 upload 152 -> 110 ms)
    const int grid = sm_count >= 8 ? sm_count / 4 : 2;
    const uintptr_t sa = (uintptr_t)src_dev_view, da = (uintptr_t)dst;
    if ((sa & 15) != (da & 15)) {
        k_copy_words<<<grid, 512, 0, s>>>((const uint32_t *)src_dev_view, (uint32_t *)dst, bytes / 4);
        return cudaGetLastError();
    }
    size_t head = (16 - (sa & 15)) & 15;            // bytes up to the first 16-byte boundary
    if (head > bytes) head = bytes;
    const size_t body = (bytes - head) & ~(size_t)15, tail = bytes - head - body;
    if (head) k_copy_words<<<1, 32, 0, s>>>((const uint32_t *)sa, (uint32_t *)da, head / 4);
    if (body)
        k_copy_vec<<<grid, 512, 0, s>>>((const uint4 *)(sa + head), (uint4 *)(da + head), body / 16);
    if (tail)
        k_copy_words<<<1, 32, 0, s>>>((const uint32_t *)(sa + head + body), (uint32_t *)(da + head + body), tail / 4);
    return cudaGetLastError();
}

}  // namespace dsg
