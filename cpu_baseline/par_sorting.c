/*
 * par_sorting.c -- a parallel CPU (OpenMP) implementation of the PaRSorting++
 * refine step (arXiv 2311.04333, Sec. 3.2-3.3 with Alg. 3), written
 * separately from the sequential oracle and from the CUDA library, for
 * timing against the GPU on the host's cores.  A CPU timing reference only: the
 * library never calls it.
 *
 * Iteration t, loads l (by id):
 *   A[u] = #{w in N(u) : (l[w], w) > (l[u], u)}      (Alg. 3, counts)
 *   order = ids sorted by (l, id): stable LSD radix sort on l - min l,
 *           8-bit digits, per-thread counts, scan, scatter
 *   B[i] = sum_{j >= i} A[order[j]]; first maximum of B[i] / (n - i)
 *           (Alg. 3, suffix densities), kept if strictly denser than the best
 *   l += A                                            (Alg. 3, load update)
 * Exact integer arithmetic; densities compared by 128-bit cross products.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

static int dens_gt(int64_t e1, int64_t v1, int64_t e2, int64_t v2)
{
    return (i128)e1 * (i128)v2 > (i128)e2 * (i128)v1;
}

/* stable LSD radix sort of ids 0..n-1 by key[id] (keys < 2^bits) */
static void radix_order(int64_t n, const uint32_t *key, int bits, uint32_t *order, uint32_t *tmp, int nt)
{
    for (int64_t i = 0; i < n; ++i) order[i] = (uint32_t)i;
    int64_t *cnt = malloc(sizeof(int64_t) * 256 * (size_t)nt);
    for (int sh = 0; sh < bits; sh += 8) {
        const int64_t chunk = (n + nt - 1) / nt;
        #pragma omp parallel num_threads(nt)
        {
            const int t = omp_get_thread_num();
            int64_t *c = cnt + 256 * t;
            memset(c, 0, sizeof(int64_t) * 256);
            const int64_t b = t * chunk, e = b + chunk < n ? b + chunk : n;
            for (int64_t i = b; i < e; ++i) c[(key[order[i]] >> sh) & 255]++;
            #pragma omp barrier
            #pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < 256; ++d)
                    for (int u = 0; u < nt; ++u) {
                        const int64_t x = cnt[256 * u + d];
                        cnt[256 * u + d] = run;
                        run += x;
                    }
            }
            for (int64_t i = b; i < e; ++i) {
                const uint32_t id = order[i];
                tmp[c[(key[id] >> sh) & 255]++] = id;
            }
        }
        memcpy(order, tmp, sizeof(uint32_t) * (size_t)n);
    }
    free(cnt);
}

/* T iterations from zero loads; loads[n] out; best = (edges, vertices,
 * iteration).  Returns 0, or 1 on allocation failure. */
int par_sorting_run(int64_t n, const int64_t *off, const int32_t *adj, int64_t T, int nthreads,
                    int64_t *loads_out, int64_t *best)
{
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
    uint32_t *l = calloc((size_t)n, 4), *A = malloc(4 * (size_t)n), *key = malloc(4 * (size_t)n);
    uint32_t *order = malloc(4 * (size_t)n), *tmp = malloc(4 * (size_t)n);
    int64_t *pre = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!l || !A || !key || !order || !tmp || !pre) return 1;
    const int64_t m = off[n] / 2;
    int64_t be = m, bv = n, bi = 0;
    for (int64_t t = 1; t <= T; ++t) {
        uint32_t lmin = UINT32_MAX, lmax = 0;
        #pragma omp parallel for num_threads(nt) schedule(dynamic, 1024) reduction(min : lmin) reduction(max : lmax)
        for (int64_t u = 0; u < n; ++u) {
            const uint32_t lu = l[u];
            uint32_t c = 0;
            for (int64_t j = off[u]; j < off[u + 1]; ++j) {
                const int32_t w = adj[j];
                c += l[w] > lu || (l[w] == lu && w > u);
            }
            A[u] = c;
            if (lu < lmin) lmin = lu;
            if (lu > lmax) lmax = lu;
        }
        const uint32_t range = lmax - lmin;
        int bits = 0;
        while (bits < 32 && (range >> bits)) bits += 8;
        #pragma omp parallel for num_threads(nt)
        for (int64_t u = 0; u < n; ++u) key[u] = l[u] - lmin;
        radix_order(n, key, bits, order, tmp, nt);
        /* suffix sums: pre[i] = sum_{j < i} A[order[j]] (chunked scan) */
        {
            const int64_t chunk = (n + nt - 1) / nt;
            int64_t *part = calloc((size_t)nt + 1, sizeof(int64_t));
            #pragma omp parallel num_threads(nt)
            {
                const int tt = omp_get_thread_num();
                const int64_t b = tt * chunk, e = b + chunk < n ? b + chunk : n;
                int64_t s = 0;
                for (int64_t i = b; i < e; ++i) s += A[order[i]];
                part[tt + 1] = s;
                #pragma omp barrier
                #pragma omp single
                for (int u = 1; u <= nt; ++u) part[u] += part[u - 1];
                int64_t run = part[tt];
                for (int64_t i = b; i < e; ++i) {
                    pre[i] = run;
                    run += A[order[i]];
                }
            }
            free(part);
        }
        /* first maximum of (m - pre[i]) / (n - i) */
        int64_t ie = m, iv = n, ipos = 0;
        #pragma omp parallel num_threads(nt)
        {
            int64_t le = -1, lv = 1, lp = -1;
            #pragma omp for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                const int64_t e = m - pre[i], v = n - i;
                if (lp < 0 || dens_gt(e, v, le, lv)) { le = e; lv = v; lp = i; }
            }
            #pragma omp critical
            {
                if (lp >= 0 && (dens_gt(le, lv, ie, iv) || (!dens_gt(ie, iv, le, lv) && lp < ipos))) {
                    ie = le; iv = lv; ipos = lp;
                }
            }
        }
        if (dens_gt(ie, iv, be, bv)) { be = ie; bv = iv; bi = t; }
        #pragma omp parallel for num_threads(nt)
        for (int64_t u = 0; u < n; ++u) l[u] += A[u];
    }
    for (int64_t u = 0; u < n; ++u) loads_out[u] = l[u];
    best[0] = be; best[1] = bv; best[2] = bi;
    free(l); free(A); free(key); free(order); free(tmp); free(pre);
    return 0;
}
