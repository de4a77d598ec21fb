/*
 * rmat_large.c -- CSR build of an R-MAT recipe (plus extra pairs such as the
 * planted blocks) that never holds the whole pair list in memory, for graphs
 * whose pair list would not fit in host RAM (scale 27: 2^31 pairs, 4.3e9
 * arcs).  The result is the same CSR as gg_build_csr gives on the full pair
 * list: symmetric, deduplicated, self-loops dropped, lists ascending, raw ids.
 *
 *   gg_large_count   -- raw arc count (with repeats) of every source vertex;
 *   gg_large_bucket  -- regenerate every pair, keep the arcs whose source lies
 *                       in [lo, hi), sort and deduplicate them and write the
 *                       lists of that source range.
 *
 * The caller cuts the source range into buckets from the raw counts, calls
 * gg_large_bucket once per bucket in increasing order and relabels after.
 * Holds no part of the densest-subgraph method: graph recipes only.
 */
#include "graphgen.h"
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* Raw arc counts: cnt[u] += 1 and cnt[v] += 1 for every pair u != v of the
 * R-MAT stream (edges 0 .. n_edges-1) and of the extra pairs. */
void gg_large_count(int scale, int64_t n_edges, uint64_t seed,
                    const uint32_t *xu, const uint32_t *xv, int64_t nx, uint32_t *cnt)
{
    uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    #pragma omp parallel for schedule(static, 1 << 16)
    for (int64_t i = 0; i < n_edges; ++i) {
        uint32_t u, v;
        gg_rmat_edge(key, scale, (uint64_t)i, &u, &v);
        if (u == v) continue;
        __atomic_fetch_add(&cnt[u], 1u, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cnt[v], 1u, __ATOMIC_RELAXED);
    }
    for (int64_t i = 0; i < nx; ++i) {
        if (xu[i] == xv[i]) continue;
        cnt[xu[i]]++;
        cnt[xv[i]]++;
    }
}

#define LOCAL_BUF 4096

static void push_local(uint64_t *buf, int64_t cap, int64_t *fill, uint64_t *loc, int *nloc,
                       uint64_t x, int *overflow)
{
    loc[(*nloc)++] = x;
    if (*nloc == LOCAL_BUF) {
        int64_t at = __atomic_fetch_add(fill, (int64_t)LOCAL_BUF, __ATOMIC_RELAXED);
        if (at + LOCAL_BUF <= cap) memcpy(buf + at, loc, sizeof(uint64_t) * LOCAL_BUF);
        else *overflow = 1;
        *nloc = 0;
    }
}

/* LSD radix sort of 64-bit keys with 16-bit digits; digits at or above
 * `bits` are skipped.  Each pass counts per thread over contiguous slices and
 * scatters in slice order, so equal digits keep their order (stable).  The
 * sorted keys end in `a`. */
static void sort_keys(uint64_t *a, uint64_t *b, int64_t n, int bits)
{
    int nthr = omp_get_max_threads();
    int64_t *cnt = calloc((size_t)nthr * 65536, sizeof(int64_t));
    uint64_t *src = a, *dst = b;
    for (int sh = 0; sh < bits; sh += 16) {
        memset(cnt, 0, sizeof(int64_t) * (size_t)nthr * 65536);
        #pragma omp parallel num_threads(nthr)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / nthr, hi = n * (t + 1) / nthr;
            int64_t *c = cnt + (size_t)t * 65536;
            for (int64_t i = lo; i < hi; ++i) c[(src[i] >> sh) & 0xFFFF]++;
            #pragma omp barrier
            #pragma omp single
            {
                int64_t s = 0;
                for (int d = 0; d < 65536; ++d)
                    for (int k = 0; k < nthr; ++k) {
                        int64_t x = cnt[(size_t)k * 65536 + d];
                        cnt[(size_t)k * 65536 + d] = s;
                        s += x;
                    }
            }
            for (int64_t i = lo; i < hi; ++i) dst[c[(src[i] >> sh) & 0xFFFF]++] = src[i];
        }
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)n);
    free(cnt);
}

/* The lists of sources lo .. hi-1: every arc (u, v) with lo <= u < hi of the
 * pairs, sorted by (u, v) and deduplicated.  buf and tmp hold `cap` keys
 * each (at least the raw arc count of the range).  adj receives the targets
 * (raw ids) list after list; deg[u - lo] the deduplicated degree.  Returns the
 * number of arcs written, or -1 if `cap` is short. */
int64_t gg_large_bucket(int scale, int64_t n_edges, uint64_t seed,
                        const uint32_t *xu, const uint32_t *xv, int64_t nx,
                        uint32_t lo, uint32_t hi, uint64_t *buf, uint64_t *tmp, int64_t cap,
                        int32_t *adj, int64_t *deg)
{
    uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    int64_t fill = 0;
    int overflow = 0;
    #pragma omp parallel
    {
        uint64_t loc[LOCAL_BUF];
        int nloc = 0, ovf = 0;
        #pragma omp for schedule(static, 1 << 16)
        for (int64_t i = 0; i < n_edges; ++i) {
            uint32_t u, v;
            gg_rmat_edge(key, scale, (uint64_t)i, &u, &v);
            if (u == v) continue;
            if (u >= lo && u < hi) push_local(buf, cap, &fill, loc, &nloc, ((uint64_t)(u - lo) << 32) | v, &ovf);
            if (v >= lo && v < hi) push_local(buf, cap, &fill, loc, &nloc, ((uint64_t)(v - lo) << 32) | u, &ovf);
        }
        if (nloc) {
            int64_t at = __atomic_fetch_add(&fill, (int64_t)nloc, __ATOMIC_RELAXED);
            if (at + nloc <= cap) memcpy(buf + at, loc, sizeof(uint64_t) * (size_t)nloc);
            else ovf = 1;
        }
        if (ovf) __atomic_store_n(&overflow, 1, __ATOMIC_RELAXED);
    }
    for (int64_t i = 0; i < nx && !overflow; ++i) {
        uint32_t u = xu[i], v = xv[i];
        if (u == v) continue;
        if (u >= lo && u < hi) { if (fill >= cap) overflow = 1; else buf[fill++] = ((uint64_t)(u - lo) << 32) | v; }
        if (v >= lo && v < hi) { if (fill >= cap) overflow = 1; else buf[fill++] = ((uint64_t)(v - lo) << 32) | u; }
    }
    if (overflow) return -1;
    int span = 0;
    while (span < 32 && ((uint64_t)1 << span) < (uint64_t)(hi - lo)) ++span;
    sort_keys(buf, tmp, fill, 32 + span);
    memset(deg, 0, sizeof(int64_t) * (size_t)(hi - lo));
    int64_t k = 0;
    for (int64_t i = 0; i < fill; ++i) {
        if (i > 0 && buf[i] == buf[i - 1]) continue;
        adj[k++] = (int32_t)(buf[i] & 0xFFFFFFFFull);
        deg[buf[i] >> 32]++;
    }
    return k;
}
