/*
 * graphgen.c -- CPU side of the seeded synthetic graph recipes (see
 * graphgen.h for the random-number definition).  Produces undirected simple
 * graphs in CSR form: symmetrised, deduplicated, self-loops removed and,
 * on request, zero-degree vertices removed with ids relabelled in their
 * original relative order.  No part of the densest-subgraph method is here.
 */
#include "graphgen.h"
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Edge list producers: each writes undirected pairs (u, v) into eu/ev (room
 * for `cap` pairs) and returns how many it wrote, or -1 if `cap` is short. */

/* G(n, p) with p = p_num / p_den: pair (i < j) is an edge iff draw
 * i*n + j of the ER stream is below floor(2^64 * p).  Plus a clique on k
 * vertices chosen by a partial Fisher-Yates shuffle of 0..n-1 whose step i
 * swaps position i with i + draw_i mod (n - i). */
int64_t gg_er_planted_clique(int64_t n, uint64_t p_num, uint64_t p_den, int64_t k,
                             uint64_t seed, uint32_t *eu, uint32_t *ev, int64_t cap)
{
    uint64_t key = gg_key(seed, GG_STREAM_ER);
    uint64_t thr = (p_num >= p_den) ? ~0ull
                 : (uint64_t)(((u128)1 << 64) * (u128)p_num / (u128)p_den);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (gg_draw(key, (uint64_t)(i * n + j)) < thr) {
                if (c >= cap) return -1;
                eu[c] = (uint32_t)i; ev[c] = (uint32_t)j; ++c;
            }
    if (k > 0) {
        uint64_t ck = gg_key(seed, GG_STREAM_CLIQUE);
        uint32_t *perm = malloc(sizeof(uint32_t) * (size_t)n);
        if (!perm) return -1;
        for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
        for (int64_t i = 0; i < k && i < n; ++i) {
            int64_t j = i + (int64_t)(gg_draw(ck, (uint64_t)i) % (uint64_t)(n - i));
            uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        for (int64_t a = 0; a < k; ++a)
            for (int64_t b = a + 1; b < k; ++b) {
                if (c >= cap) { free(perm); return -1; }
                eu[c] = perm[a]; ev[c] = perm[b]; ++c;
            }
        free(perm);
    }
    return c;
}

/* R-MAT edges 0 .. n_edges-1 at `scale` (see gg_rmat_edge). */
int64_t gg_rmat(int scale, int64_t n_edges, uint64_t seed,
                uint32_t *eu, uint32_t *ev, int64_t cap)
{
    if (n_edges > cap) return -1;
    uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    for (int64_t i = 0; i < n_edges; ++i)
        gg_rmat_edge(key, scale, (uint64_t)i, &eu[i], &ev[i]);
    return n_edges;
}

/* The affine permutation of planted blocks (see gg_block_vertex). */
void gg_block_perm(uint64_t seed, uint64_t *mul, uint64_t *add)
{
    uint64_t key = gg_key(seed, GG_STREAM_BLOCK_PERM);
    *mul = gg_draw(key, 0) | 1ull;
    *add = gg_draw(key, 1);
}

/* Planted G(s_b, 1/2) blocks appended after `start` existing pairs. */
int64_t gg_planted_blocks(int scale, int nblocks, const int64_t *sizes, uint64_t seed,
                          uint32_t *eu, uint32_t *ev, int64_t start, int64_t cap)
{
    uint64_t mul, add;
    gg_block_perm(seed, &mul, &add);
    int64_t c = start, base = 0;
    for (int b = 0; b < nblocks; ++b) {
        int64_t s = sizes[b];
        uint64_t key = gg_key(seed, GG_STREAM_BLOCK_EDGES + (uint64_t)b);
        for (int64_t i = 0; i < s; ++i)
            for (int64_t j = i + 1; j < s; ++j)
                if ((gg_draw(key, (uint64_t)(i * s + j)) >> 63) == 0) {
                    if (c >= cap) return -1;
                    eu[c] = gg_block_vertex(mul, add, scale, (uint64_t)(base + i));
                    ev[c] = gg_block_vertex(mul, add, scale, (uint64_t)(base + j));
                    ++c;
                }
        base += s;
    }
    return c;
}

/* G(n, M)-style random graph: M draws of a pair (draw 2e mod n, draw 2e+1
 * mod n); self-loops and repeats are removed later by the CSR build. */
int64_t gg_er_m(int64_t n, int64_t M, uint64_t seed, uint32_t *eu, uint32_t *ev, int64_t cap)
{
    if (M > cap) return -1;
    uint64_t key = gg_key(seed, GG_STREAM_ER);
    for (int64_t e = 0; e < M; ++e) {
        eu[e] = (uint32_t)(gg_draw(key, 2 * (uint64_t)e) % (uint64_t)n);
        ev[e] = (uint32_t)(gg_draw(key, 2 * (uint64_t)e + 1) % (uint64_t)n);
    }
    return M;
}

/* Chung-Lu style power-law graph: integer weights w_i (given by the caller,
 * non-increasing), M edges whose endpoints are drawn independently with
 * probability proportional to w (inverse-CDF search on the prefix sums). */
int64_t gg_weighted_pairs(int64_t n, const uint64_t *cum_w, int64_t M, uint64_t seed,
                          uint32_t *eu, uint32_t *ev, int64_t cap)
{
    if (M > cap || n < 1) return -1;
    uint64_t key = gg_key(seed, GG_STREAM_ER);
    uint64_t total = cum_w[n - 1];
    for (int64_t e = 0; e < M; ++e) {
        for (int side = 0; side < 2; ++side) {
            uint64_t x = gg_draw(key, 2 * (uint64_t)e + (uint64_t)side) % total;
            int64_t lo = 0, hi = n - 1;          /* first i with cum_w[i] > x */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (cum_w[mid] > x) hi = mid; else lo = mid + 1;
            }
            if (side == 0) eu[e] = (uint32_t)lo; else ev[e] = (uint32_t)lo;
        }
    }
    return M;
}

/* LSD radix sort of 64-bit keys, 16-bit digits, skipping constant digits. */
static int radix_sort_u64(uint64_t *a, int64_t n)
{
    uint64_t *b = malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    int64_t *cnt = malloc(sizeof(int64_t) * 65536);
    if (!b || !cnt) { free(b); free(cnt); return -1; }
    for (int d = 0; d < 4; ++d) {
        int sh = 16 * d;
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t i = 0; i < n; ++i) cnt[(a[i] >> sh) & 0xFFFF]++;
        int nonzero = 0;
        for (int i = 0; i < 65536; ++i) nonzero += cnt[i] != 0;
        if (nonzero <= 1) continue;
        int64_t s = 0;
        for (int i = 0; i < 65536; ++i) { int64_t c = cnt[i]; cnt[i] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) b[cnt[(a[i] >> sh) & 0xFFFF]++] = a[i];
        memcpy(a, b, sizeof(uint64_t) * (size_t)n);
    }
    free(b); free(cnt);
    return 0;
}

/* Build the CSR of the simple undirected graph on ids 0..n_raw-1 given by
 * the pairs: both directions, duplicates and self-loops dropped, adjacency
 * lists ascending.  If drop_isolated, zero-degree vertices are removed and
 * the rest relabelled in increasing original id; new_id (optional, n_raw)
 * receives the new id or -1.  off_out needs n_raw+1 entries, adj_out 2*E.
 * Returns the number of vertices kept; *arcs_out receives off[n]. */
int64_t gg_build_csr(int64_t n_raw, int64_t E, const uint32_t *eu, const uint32_t *ev,
                     int drop_isolated, int64_t *off_out, int32_t *adj_out,
                     int64_t *new_id, int64_t *arcs_out)
{
    uint64_t *arc = malloc(sizeof(uint64_t) * (size_t)(2 * E + 1));
    int64_t *deg = calloc((size_t)n_raw + 1, sizeof(int64_t));
    int64_t *nid = malloc(sizeof(int64_t) * (size_t)(n_raw + 1));
    if (!arc || !deg || !nid) { free(arc); free(deg); free(nid); return -1; }
    int64_t na = 0;
    for (int64_t e = 0; e < E; ++e) {
        if (eu[e] == ev[e]) continue;
        arc[na++] = ((uint64_t)eu[e] << 32) | ev[e];
        arc[na++] = ((uint64_t)ev[e] << 32) | eu[e];
    }
    if (radix_sort_u64(arc, na)) { free(arc); free(deg); free(nid); return -1; }
    int64_t k = 0;
    for (int64_t i = 0; i < na; ++i)
        if (i == 0 || arc[i] != arc[i - 1]) arc[k++] = arc[i];
    na = k;
    for (int64_t i = 0; i < na; ++i) deg[arc[i] >> 32]++;
    int64_t nk = 0;
    for (int64_t v = 0; v < n_raw; ++v)
        nid[v] = (!drop_isolated || deg[v] > 0) ? nk++ : -1;
    off_out[0] = 0;
    int64_t o = 0;
    for (int64_t v = 0; v < n_raw; ++v)
        if (nid[v] >= 0) { o += deg[v]; off_out[nid[v] + 1] = o; }
    for (int64_t i = 0; i < na; ++i)
        adj_out[i] = (int32_t)nid[arc[i] & 0xFFFFFFFFull];
    if (new_id) memcpy(new_id, nid, sizeof(int64_t) * (size_t)n_raw);
    *arcs_out = na;
    free(arc); free(deg); free(nid);
    return nk;
}
