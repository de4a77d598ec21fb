/*
 * oracle.c -- plain, slow, sequential CPU oracle for the load-weighted peeling
 * of Greedy++ (arXiv 2311.04333) in its sorting form (GreedySorting++, the
 * ordering behind PaRSorting++) and its round-peeling form (ParallelGreedy++,
 * the ordering behind PaRGreedy++).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * link it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is exact integer arithmetic.  Densities are (edges, vertices)
 * pairs compared by cross-multiplication in 128 bits.
 *
 * Structure (each function names the passage it follows):
 *   - ordering functions O (Alg. 2, order of each iteration): sort by load (Sec. 3.2,
 *     "GreedySorting++"), simultaneous round peeling (Sec. 3.3,
 *     "ParallelGreedy++"), and the one-at-a-time load ordering (Sec. 2,
 *     "load ordering"; Greedy++ proper);
 *   - the peel of one iteration in that order, one vertex at a time, exactly
 *     as Alg. 2's inner loop states it (density check, load += induced degree at
 *     peel time, remove the vertex).  This is deliberately NOT Alg. 3's
 *     parallel A[min(j,k)] formulation, so the GPU's Alg. 3 path is checked
 *     against the sequential definition;
 *   - Alg. 1 (Pruning-and-Refining) with exact pruning, or with pruning by
 *     a c-approximate k-core decomposition (Sec. 2 definition, Sec. 4
 *     approximate variants) taken at geometric levels of the core numbers;
 *   - exact checkers used to pin the oracle: brute force over all subsets,
 *     Goldberg-style max-flow densest subgraph, Batagelj-Zaversnik coreness,
 *     and the textbook k-core by repeated deletion (Sec. 2, Definitions of
 *     k-core and core number).
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   - ties in the load sort are broken by ascending vertex id;
 *   - H is reset to G at the start of every iteration (Alg. 2 writes H <- G
 *     once, before the loop; peeling an empty H afterwards would be vacuous);
 *   - within one ParallelGreedy++ round the peeled vertices are ordered by
 *     ascending id, so deg* of a vertex is its number of neighbours later in
 *     the (round, id) order;
 *   - a round peels every alive v with key(v)*q <= min_key*(p+q), eps = p/q
 *     (eps = 0 is the paper's exact bucket peel of the minimum key only);
 *   - the best subgraph starts as S = G and is replaced only on a strictly
 *     higher density (Alg. 2: S starts as G, strict test), so ties keep the earliest
 *     (iteration, position); the empty suffix is never a candidate.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_NOMEM 2

/* rho(e1/v1) > rho(e2/v2) with v1, v2 > 0 (Sec. 2: rho(G) = |E|/|V|). */
static int density_gt(int64_t e1, int64_t v1, int64_t e2, int64_t v2)
{
    return (i128)e1 * (i128)v2 > (i128)e2 * (i128)v1;
}

/* ------------------------------------------------------------------------ */
/* Ordering O for GreedySorting++ (Sec. 3.2): l(v_1) <= ... <= l(v_n), ties
 * by vertex id.  A library sort (qsort) on the total order (load, id).      */

static const int64_t *g_sort_loads;

static int cmp_load_id(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    int64_t lx = g_sort_loads[x], ly = g_sort_loads[y];
    if (lx != ly) return lx < ly ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_sorting_order(int64_t n, const int64_t *loads, int64_t *order)
{
    if (n < 0) return OR_ERR_INVALID;
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_loads = loads;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_load_id);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Ordering O for ParallelGreedy++ (Sec. 3.3): bucketed peeling by the key
 * l(v) + deg_H(v).  Each round takes every alive vertex whose key is within a
 * (1 + p/q) factor of the current minimum key, appends them in ascending id,
 * and only then applies their degree decrements to the vertices that stay
 * alive ("this effect is delayed until the end of the peeling step").
 * round_of[v] receives the round index (may be NULL); returns the number of
 * rounds (the peeling complexity c_p of this iteration), or -1 on error.    */
int64_t oracle_round_order(int64_t n, const int64_t *off, const int32_t *adj,
                           const int64_t *loads, int64_t p, int64_t q,
                           int64_t *order, int64_t *round_of, int64_t *round_min)
{
    if (n < 0 || q <= 0 || p < 0) return -1;
    int64_t *deg = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *alive = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    unsigned char *state = calloc((size_t)(n ? n : 1), 1); /* 0 alive, 1 in F, 2 peeled */
    if (!deg || !alive || !state) { free(deg); free(alive); free(state); return -1; }
    for (int64_t v = 0; v < n; ++v) { deg[v] = off[v + 1] - off[v]; alive[v] = v; }
    int64_t n_alive = n, pos = 0, r = 0;
    while (n_alive > 0) {
        int64_t mn = INT64_MAX;
        for (int64_t i = 0; i < n_alive; ++i) {
            int64_t v = alive[i];
            int64_t k = loads[v] + deg[v];
            if (k < mn) mn = k;
        }
        if (round_min) round_min[r] = mn;
        int64_t start = pos, keep = 0;
        for (int64_t i = 0; i < n_alive; ++i) {   /* alive[] stays in id order */
            int64_t v = alive[i];
            int64_t k = loads[v] + deg[v];
            if ((i128)k * q <= (i128)mn * (i128)(p + q)) {
                order[pos++] = v;
                state[v] = 1;
                if (round_of) round_of[v] = r;
            } else {
                alive[keep++] = v;
            }
        }
        for (int64_t j = start; j < pos; ++j) {
            int64_t v = order[j];
            for (int64_t e = off[v]; e < off[v + 1]; ++e)
                if (state[adj[e]] == 0) deg[adj[e]] -= 1;
        }
        for (int64_t j = start; j < pos; ++j) state[order[j]] = 2;
        n_alive = keep;
        ++r;
    }
    free(deg); free(alive); free(state);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Ordering O for sequential Greedy++ (Sec. 2 "load ordering", Sec. 3.2):
 * repeatedly peel the vertex minimising l(v) + deg_H(v) (ties: smallest id),
 * one vertex at a time, degrees updated immediately.  O(n^2): small inputs. */
int oracle_load_order(int64_t n, const int64_t *off, const int32_t *adj,
                      const int64_t *loads, int64_t *order)
{
    int64_t *deg = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    unsigned char *gone = calloc((size_t)(n ? n : 1), 1);
    if (!deg || !gone) { free(deg); free(gone); return OR_ERR_NOMEM; }
    for (int64_t v = 0; v < n; ++v) deg[v] = off[v + 1] - off[v];
    for (int64_t j = 0; j < n; ++j) {
        int64_t best = -1, bk = 0;
        for (int64_t v = 0; v < n; ++v) {
            if (gone[v]) continue;
            int64_t k = loads[v] + deg[v];
            if (best < 0 || k < bk) { best = v; bk = k; }
        }
        order[j] = best;
        gone[best] = 1;
        for (int64_t e = off[best]; e < off[best + 1]; ++e)
            if (!gone[adj[e]]) deg[adj[e]] -= 1;
    }
    free(deg); free(gone);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* One iteration of Alg. 2's inner loop for a given order v_1..v_n, with H
 * reset to G: for j = 1..n, if rho(H) > rho(best) then best <- H; then
 * l(v_j) += deg*_H(v_j) (degree of v_j in H when it is peeled) and peel v_j.
 *
 * degstar[j] receives deg*_H(v_j) (this is A[j] of Alg. 3).
 * it_best[0..2] receives the densest suffix of this iteration alone
 *   (edges, vertices, position j of its first vertex), first one on ties.
 * *best_e / *best_v hold the running best; *improved_at receives the
 *   position j at which the running best was last replaced in this
 *   iteration, or -1.  width receives max_j deg*_H(v_j).                   */
int oracle_peel_iteration(int64_t n, const int64_t *off, const int32_t *adj,
                          const int64_t *order, int64_t *loads,
                          int64_t *degstar, int64_t *it_best,
                          int64_t *best_e, int64_t *best_v,
                          int64_t *improved_at, int64_t *width)
{
    int64_t *deg = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    unsigned char *inH = malloc((size_t)(n ? n : 1));
    if (!deg || !inH) { free(deg); free(inH); return OR_ERR_NOMEM; }
    int64_t eH = 0;
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        eH += deg[v];
        inH[v] = 1;
    }
    eH /= 2;
    int64_t vH = n;
    int64_t ie = -1, iv = 1, ij = -1, w = 0;
    *improved_at = -1;
    for (int64_t j = 0; j < n; ++j) {
        int64_t v = order[j];
        /* this iteration's own densest suffix: first maximum */
        if (ij < 0 || density_gt(eH, vH, ie, iv)) { ie = eH; iv = vH; ij = j; }
        /* Alg. 2: the running best, strict comparison */
        if (density_gt(eH, vH, *best_e, *best_v)) {
            *best_e = eH; *best_v = vH; *improved_at = j;
        }
        int64_t ds = deg[v];                 /* deg*_H(v_j) */
        degstar[j] = ds;
        if (ds > w) w = ds;
        loads[v] += ds;                      /* Alg. 2: load update */
        inH[v] = 0;                          /* Alg. 2: peel v */
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (inH[adj[e]]) deg[adj[e]] -= 1;
        eH -= ds;
        vH -= 1;
    }
    if (it_best) { it_best[0] = ie < 0 ? 0 : ie; it_best[1] = ie < 0 ? 0 : iv; it_best[2] = ij; }
    if (width) *width = w;
    free(deg); free(inH);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* T iterations of Alg. 2 with the chosen ordering function.
 *   variant 0: GreedySorting++ order (PaRSorting++ refine step)
 *   variant 1: ParallelGreedy++ round order with eps = p/q (PaRGreedy++)
 *   variant 2: sequential Greedy++ load order
 * init_loads may be NULL (Alg. 2 starts from l = 0).  On return loads[n]
 * holds the final loads, best_e/best_v/best_iter the best density (iteration
 * 0 means S = G was never beaten), set[] the best subgraph's vertex ids in
 * ascending order (set_size of them), and trace[3*t..3*t+2] (if not NULL)
 * the densest suffix of iteration t+1 (edges, vertices) and its width.
 * best_pos receives the position of the best suffix in its iteration.      */
int oracle_run(int64_t n, const int64_t *off, const int32_t *adj,
               int variant, int64_t T, int64_t p, int64_t q,
               const int64_t *init_loads, int64_t *loads,
               int64_t *best, int64_t *set, int64_t *trace)
{
    if (n < 1 || T < 0 || q <= 0 || p < 0 || variant < 0 || variant > 2)
        return OR_ERR_INVALID;
    int64_t *order = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *border = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *degstar = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *start = malloc(sizeof(int64_t) * (size_t)n);
    if (!order || !border || !degstar || !start) {
        free(order); free(border); free(degstar); free(start);
        return OR_ERR_NOMEM;
    }
    for (int64_t v = 0; v < n; ++v) loads[v] = init_loads ? init_loads[v] : 0;
    int64_t m = off[n] / 2;
    int64_t be = m, bv = n, biter = 0, bpos = 0;        /* S <- G (Alg. 2) */
    for (int64_t t = 1; t <= T; ++t) {
        memcpy(start, loads, sizeof(int64_t) * (size_t)n);
        if (variant == 0) oracle_sorting_order(n, start, order);
        else if (variant == 1) {
            if (oracle_round_order(n, off, adj, start, p, q, order, NULL, NULL) < 0) {
                free(order); free(border); free(degstar); free(start);
                return OR_ERR_NOMEM;
            }
        } else oracle_load_order(n, off, adj, start, order);
        int64_t it_best[3], at = -1, w = 0;
        oracle_peel_iteration(n, off, adj, order, loads, degstar, it_best,
                              &be, &bv, &at, &w);
        if (at >= 0) {
            biter = t; bpos = at;
            memcpy(border, order, sizeof(int64_t) * (size_t)n);
        }
        if (trace) {
            trace[3 * (t - 1) + 0] = it_best[0];
            trace[3 * (t - 1) + 1] = it_best[1];
            trace[3 * (t - 1) + 2] = w;
        }
    }
    /* best subgraph as ascending ids */
    int64_t k = 0;
    if (biter == 0) {
        for (int64_t v = 0; v < n; ++v) set[k++] = v;
    } else {
        unsigned char *in = calloc((size_t)n, 1);
        if (!in) { free(order); free(border); free(degstar); free(start); return OR_ERR_NOMEM; }
        for (int64_t j = bpos; j < n; ++j) in[border[j]] = 1;
        for (int64_t v = 0; v < n; ++v) if (in[v]) set[k++] = v;
        free(in);
    }
    best[0] = be; best[1] = bv; best[2] = biter; best[3] = k; best[4] = bpos;
    free(order); free(border); free(degstar); free(start);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact checkers used to pin the oracle.                                    */

/* Brute force over all 2^n - 1 non-empty vertex subsets (n <= 24): the
 * densest subgraph by its definition (Sec. 2).  First subset in increasing
 * bitmask order among the densest; returns (edges, vertices, mask).        */
int oracle_brute_force(int64_t n, const int64_t *off, const int32_t *adj,
                       int64_t *out)
{
    if (n < 1 || n > 24) return OR_ERR_INVALID;
    uint32_t nb[24];
    for (int64_t v = 0; v < n; ++v) {
        nb[v] = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) nb[v] |= 1u << adj[e];
    }
    int64_t be = 0, bv = 1, bm = 0;
    uint32_t full = (n == 32) ? 0xffffffffu : ((1u << n) - 1u);
    for (uint32_t S = 1; S <= full && S != 0; ++S) {
        int64_t twice = 0, vs = 0;
        for (int64_t v = 0; v < n; ++v)
            if (S >> v & 1u) { ++vs; twice += __builtin_popcount(nb[v] & S); }
        if (bm == 0 || density_gt(twice / 2, vs, be, bv)) { be = twice / 2; bv = vs; bm = S; }
        if (S == full) break;
    }
    out[0] = be; out[1] = bv; out[2] = bm;
    return OR_OK;
}

/* Dinic max-flow on a small network, int64 capacities. */
typedef struct { int64_t to, cap, next; } arc_t;
typedef struct {
    int64_t nv, na, cap_arcs;
    arc_t *a;
    int64_t *head, *level, *it, *queue;
} flow_t;

static int flow_init(flow_t *f, int64_t nv, int64_t max_arcs)
{
    f->nv = nv; f->na = 0; f->cap_arcs = max_arcs;
    f->a = malloc(sizeof(arc_t) * (size_t)max_arcs);
    f->head = malloc(sizeof(int64_t) * (size_t)nv);
    f->level = malloc(sizeof(int64_t) * (size_t)nv);
    f->it = malloc(sizeof(int64_t) * (size_t)nv);
    f->queue = malloc(sizeof(int64_t) * (size_t)nv);
    if (!f->a || !f->head || !f->level || !f->it || !f->queue) return -1;
    for (int64_t i = 0; i < nv; ++i) f->head[i] = -1;
    return 0;
}
static void flow_free(flow_t *f)
{
    free(f->a); free(f->head); free(f->level); free(f->it); free(f->queue);
}
static void flow_add(flow_t *f, int64_t u, int64_t v, int64_t c)
{
    f->a[f->na] = (arc_t){v, c, f->head[u]}; f->head[u] = f->na++;
    f->a[f->na] = (arc_t){u, 0, f->head[v]}; f->head[v] = f->na++;
}
static int flow_bfs(flow_t *f, int64_t s, int64_t t)
{
    for (int64_t i = 0; i < f->nv; ++i) f->level[i] = -1;
    int64_t qh = 0, qt = 0;
    f->queue[qt++] = s; f->level[s] = 0;
    while (qh < qt) {
        int64_t u = f->queue[qh++];
        for (int64_t e = f->head[u]; e >= 0; e = f->a[e].next)
            if (f->a[e].cap > 0 && f->level[f->a[e].to] < 0) {
                f->level[f->a[e].to] = f->level[u] + 1;
                f->queue[qt++] = f->a[e].to;
            }
    }
    return f->level[t] >= 0;
}
/* iterative blocking-flow DFS */
static int64_t flow_dfs(flow_t *f, int64_t s, int64_t t)
{
    int64_t total = 0;
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)f->nv);   /* arcs on path */
    for (;;) {
        int64_t depth = 0, u = s;
        for (;;) {
            if (u == t) {
                int64_t push = INT64_MAX;
                for (int64_t i = 0; i < depth; ++i)
                    if (f->a[stack[i]].cap < push) push = f->a[stack[i]].cap;
                for (int64_t i = 0; i < depth; ++i) {
                    f->a[stack[i]].cap -= push;
                    f->a[stack[i] ^ 1].cap += push;
                }
                total += push;
                depth = 0; u = s;
                continue;
            }
            int64_t e;
            for (e = f->it[u]; e >= 0; e = f->a[e].next)
                if (f->a[e].cap > 0 && f->level[f->a[e].to] == f->level[u] + 1) break;
            f->it[u] = e;
            if (e >= 0) {
                stack[depth++] = e;
                u = f->a[e].to;
            } else {
                if (depth == 0) { free(stack); return total; }
                f->level[u] = -1;                 /* dead end */
                int64_t back = stack[--depth];
                u = f->a[back ^ 1].to;
                f->it[u] = f->a[f->it[u]].next;
            }
        }
    }
}
static int64_t flow_max(flow_t *f, int64_t s, int64_t t)
{
    int64_t total = 0;
    while (flow_bfs(f, s, t)) {
        for (int64_t i = 0; i < f->nv; ++i) f->it[i] = f->head[i];
        total += flow_dfs(f, s, t);
    }
    return total;
}

/* Exact densest subgraph by parametric min cut (the flow approach the paper
 * cites for exact solutions, Sec. 1 and Sec. 3).  For a guess g = a/b the
 * maximum of b|E(S)| - a|V(S)| over vertex sets S is m*b - mincut of the
 * network  s -> edge node (cap b),  edge node -> both endpoints (cap inf),
 * vertex -> t (cap a)  (the selection / closure problem).  Starting from
 * g = rho(G), a positive maximum yields a set S' of higher density; repeat
 * with g = rho(S') (Dinkelbach) until the maximum is 0, at which point
 * g = rho*.  out = (edges, vertices) of rho*; set_out (optional, n bytes)
 * marks a densest subgraph.                                                  */
int oracle_maxflow_densest(int64_t n, const int64_t *off, const int32_t *adj,
                           int64_t *out, unsigned char *set_out)
{
    if (n < 1) return OR_ERR_INVALID;
    int64_t m = off[n] / 2;
    if (m == 0) {
        out[0] = 0; out[1] = n;
        if (set_out) for (int64_t v = 0; v < n; ++v) set_out[v] = 1;
        return OR_OK;
    }
    int64_t *eu = malloc(sizeof(int64_t) * (size_t)m), *ev = malloc(sizeof(int64_t) * (size_t)m);
    unsigned char *side = malloc((size_t)n);
    if (!eu || !ev || !side) { free(eu); free(ev); free(side); return OR_ERR_NOMEM; }
    int64_t k = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            if (adj[e] > u) { eu[k] = u; ev[k] = adj[e]; ++k; }
    int64_t ga = m, gb = n;                     /* g = rho(G) */
    for (int v = 0; v < n; ++v) side[v] = 1;
    const int64_t INF = (int64_t)1 << 60;
    for (int rounds = 0; rounds < 10000; ++rounds) {
        flow_t f;
        int64_t s = n + m, t = n + m + 1;
        if (flow_init(&f, n + m + 2, 2 * (m + 2 * m + n))) { flow_free(&f); free(eu); free(ev); free(side); return OR_ERR_NOMEM; }
        for (int64_t i = 0; i < m; ++i) {
            flow_add(&f, s, n + i, gb);
            flow_add(&f, n + i, eu[i], INF);
            flow_add(&f, n + i, ev[i], INF);
        }
        for (int64_t v = 0; v < n; ++v) flow_add(&f, v, t, ga);
        int64_t cut = flow_max(&f, s, t);
        int64_t val = m * gb - cut;             /* max_S b|E(S)| - a|V(S)| */
        if (val <= 0) { flow_free(&f); break; }
        /* source side of the min cut: reachable from s in the residual graph */
        flow_bfs(&f, s, t);
        int64_t vs = 0, es = 0;
        for (int64_t v = 0; v < n; ++v) { side[v] = f.level[v] >= 0; vs += side[v]; }
        for (int64_t i = 0; i < m; ++i) es += side[eu[i]] && side[ev[i]];
        flow_free(&f);
        ga = es; gb = vs;
    }
    out[0] = ga; out[1] = gb;
    if (set_out) for (int64_t v = 0; v < n; ++v) set_out[v] = side[v];
    free(eu); free(ev); free(side);
    return OR_OK;
}

/* Core numbers by the Batagelj-Zaversnik bin-sort algorithm (O(m)):
 * process vertices in non-decreasing current degree; each processed vertex
 * fixes its core number and lowers the degree of unprocessed neighbours
 * whose degree is larger (Sec. 2, Definition of core number).              */
int oracle_coreness(int64_t n, const int64_t *off, const int32_t *adj, int64_t *core)
{
    int64_t md = 0;
    int64_t *deg = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *vert = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *pos = malloc(sizeof(int64_t) * (size_t)n);
    if (!deg || !vert || !pos) { free(deg); free(vert); free(pos); return OR_ERR_NOMEM; }
    for (int64_t v = 0; v < n; ++v) { deg[v] = off[v + 1] - off[v]; if (deg[v] > md) md = deg[v]; }
    int64_t *bin = calloc((size_t)(md + 2), sizeof(int64_t));
    if (!bin) { free(deg); free(vert); free(pos); return OR_ERR_NOMEM; }
    for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
    int64_t s = 0;
    for (int64_t d = 0; d <= md; ++d) { int64_t c = bin[d]; bin[d] = s; s += c; }
    for (int64_t v = 0; v < n; ++v) { pos[v] = bin[deg[v]]; vert[pos[v]] = v; bin[deg[v]]++; }
    for (int64_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = vert[i];
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int64_t u = adj[e];
            if (deg[u] > deg[v]) {
                int64_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) core[v] = deg[v];
    free(deg); free(vert); free(pos); free(bin);
    return OR_OK;
}

/* k-core by its definition (Sec. 2): for each k, repeatedly delete vertices
 * of degree < k; core(v) is the largest k for which v survives.  O(n m k). */
int oracle_coreness_by_deletion(int64_t n, const int64_t *off, const int32_t *adj, int64_t *core)
{
    unsigned char *in = malloc((size_t)n);
    if (!in) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; ++v) core[v] = 0;
    for (int64_t k = 1;; ++k) {
        for (int64_t v = 0; v < n; ++v) in[v] = 1;
        int changed = 1;
        while (changed) {
            changed = 0;
            for (int64_t v = 0; v < n; ++v) {
                if (!in[v]) continue;
                int64_t d = 0;
                for (int64_t e = off[v]; e < off[v + 1]; ++e) d += in[adj[e]];
                if (d < k) { in[v] = 0; changed = 1; }
            }
        }
        int any = 0;
        for (int64_t v = 0; v < n; ++v) if (in[v]) { core[v] = k; any = 1; }
        if (!any) break;
    }
    free(in);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Pruning-and-Refining framework (Alg. 1, Sec. 3) with exact pruning.      */

/* getCore (Alg. 1, initial and re-pruning): the subgraph of G induced on the vertices
 * with in[v] != 0, relabelled in increasing id (lists keep their order).
 * old_of[local] = original id.                                             */
static int induced_subgraph(int64_t n, const int64_t *off, const int32_t *adj, const unsigned char *in,
                            int64_t *nn_out, int64_t **off_out, int32_t **adj_out, int64_t **old_of_out)
{
    int64_t *new_id = malloc(sizeof(int64_t) * (size_t)n);
    if (!new_id) return OR_ERR_NOMEM;
    int64_t nn = 0;
    for (int64_t v = 0; v < n; ++v) new_id[v] = in[v] ? nn++ : -1;
    int64_t *noff = malloc(sizeof(int64_t) * (size_t)(nn + 1));
    int64_t *old_of = malloc(sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
    if (!noff || !old_of) { free(new_id); free(noff); free(old_of); return OR_ERR_NOMEM; }
    int64_t arcs = 0;
    noff[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (!in[v]) continue;
        old_of[new_id[v]] = v;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) arcs += in[adj[e]] ? 1 : 0;
        noff[new_id[v] + 1] = arcs;
    }
    int32_t *nadj = malloc(sizeof(int32_t) * (size_t)(arcs > 0 ? arcs : 1));
    if (!nadj) { free(new_id); free(noff); free(old_of); return OR_ERR_NOMEM; }
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (!in[v]) continue;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (in[adj[e]]) nadj[k++] = (int32_t)new_id[adj[e]];
    }
    free(new_id);
    *nn_out = nn; *off_out = noff; *adj_out = nadj; *old_of_out = old_of;
    return OR_OK;
}

/* ceil(a / b) for a >= 0, b > 0 */
static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* The k-core of G for the given core numbers: the induced subgraph on
 * {v : core(v) >= k} (exported for the pins of Lemma "core contains S*"). */
int oracle_core_subgraph(int64_t n, const int64_t *off, const int32_t *adj, const int64_t *core, int64_t k,
                         int64_t *nn, int64_t *mm)
{
    unsigned char *in = malloc((size_t)n);
    if (!in) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; ++v) in[v] = core[v] >= k;
    int64_t *o = NULL, *old_of = NULL;
    int32_t *a = NULL;
    int rc = induced_subgraph(n, off, adj, in, nn, &o, &a, &old_of);
    if (rc == OR_OK) *mm = o[*nn] / 2;
    free(in); free(o); free(a); free(old_of);
    return rc;
}

/* c-approximate k-core decomposition (Sec. 2, Def. of the c-approximate
 * decomposition; c = c_num / c_den > 1), at geometric levels
 * tau_0 = 1, tau_{i+1} = ceil(tau_i * c): a vertex of core number k >= 1
 * gets the smallest level >= k, a vertex of core number 0 gets 0.  Since
 * tau_{i+1} < c * tau_i + 1 <= c * k for k > tau_i, this k-hat satisfies
 * k <= k-hat < c * k, inside the definition's bounds k / c <= k-hat <= c k.
 * It is what peeling with the thresholds tau_i yields: the vertices left
 * after removing, level by level, every vertex of degree <= tau_i are the
 * (tau_i + 1)-core, and those removed at level i have k in (tau_{i-1}, tau_i]. */
static int64_t apx_next_level(int64_t tau, int64_t c_num, int64_t c_den)
{
    return ceil_div(tau * c_num, c_den);
}

int oracle_apx_coreness(int64_t n, const int64_t *off, const int32_t *adj, int64_t c_num, int64_t c_den,
                        int64_t *apx)
{
    if (n < 1 || c_den < 1 || c_num <= c_den) return OR_ERR_INVALID;
    int rc = oracle_coreness(n, off, adj, apx);
    if (rc != OR_OK) return rc;
    for (int64_t v = 0; v < n; ++v) {
        if (apx[v] == 0) continue;
        int64_t tau = 1;
        while (tau < apx[v]) tau = apx_next_level(tau, c_num, c_den);
        apx[v] = tau;
    }
    return OR_OK;
}

/* Alg. 1: cores <- Coreness(G); L <- ceil(k_max / 2); G <- L-core; S <- G;
 * then T times: S' <- Refine(G) (one iteration of the refine step
 * `variant` on the current G, with the loads of its vertices carried over
 * from the previous iterations); if rho(S') > rho(S): S <- S',
 * L <- max(L, rho(S)) and G <- ceil(L)-core (of the core numbers of the
 * input).  L is kept as an exact rational.
 * Outputs (original ids): loads[n] = the load of each vertex when it left G
 * (0 if never in the first core; the final loads for the final G);
 * best = (edges, vertices, iteration of the last improvement (0: the first
 * core itself), set size, 0); set = S ascending; trace[3 t ..] = (edges,
 * vertices) of the refine result of iteration t+1 and the vertex count of
 * the G it ran on; info = (k_max, |V|, |E| of the first core, |V| of the
 * final G, L as numerator, denominator).                                  */
/* With c_num > 0 the same loop runs on the c-approximate decomposition
 * above (c = c_num / c_den, approximate pruning of Sec. 4): core numbers
 * become k-hat, k_max becomes k-hat_max, the initial bound is
 * L = ceil(k-hat_max / (2 c)) (Cor. of the approximate k_max), and every
 * getCore keeps {v : k-hat(v) >= level}; info[0] is then k-hat_max.        */
int oracle_run_pruned_c(int64_t n, const int64_t *off, const int32_t *adj, int variant, int64_t T,
                        int64_t p, int64_t q, int64_t c_num, int64_t c_den, int64_t *loads, int64_t *best,
                        int64_t *set, int64_t *trace, int64_t *info)
{
    if (n < 1 || T < 0 || q <= 0 || p < 0 || variant < 0 || variant > 2) return OR_ERR_INVALID;
    if (c_num != 0 && (c_den < 1 || c_num <= c_den)) return OR_ERR_INVALID;
    int64_t *core = malloc(sizeof(int64_t) * (size_t)n);
    unsigned char *in = malloc((size_t)n);
    if (!core || !in) { free(core); free(in); return OR_ERR_NOMEM; }
    int rc = c_num ? oracle_apx_coreness(n, off, adj, c_num, c_den, core) : oracle_coreness(n, off, adj, core);
    if (rc != OR_OK) { free(core); free(in); return rc; }
    int64_t kmax = 0;
    for (int64_t v = 0; v < n; ++v) if (core[v] > kmax) kmax = core[v];
    /* Alg. 1: L = ceil(k_max / 2), or ceil(k-hat_max / (2c)) */
    int64_t Ln = c_num ? ceil_div(kmax * c_den, 2 * c_num) : ceil_div(kmax, 2), Ld = 1;
    int64_t level = Ln;
    for (int64_t v = 0; v < n; ++v) in[v] = core[v] >= level;
    int64_t cn = 0, *coff = NULL, *old_of = NULL;
    int32_t *cadj = NULL;
    rc = induced_subgraph(n, off, adj, in, &cn, &coff, &cadj, &old_of);   /* G <- L-core */
    if (rc != OR_OK) { free(core); free(in); return rc; }
    for (int64_t v = 0; v < n; ++v) loads[v] = 0;
    int64_t se = coff[cn] / 2, sv = cn, biter = 0, ssize = cn;          /* S <- G */
    for (int64_t i = 0; i < cn; ++i) set[i] = old_of[i];
    if (info) { info[0] = kmax; info[1] = cn; info[2] = coff[cn] / 2; }
    int64_t *cl = calloc((size_t)(cn > 0 ? cn : 1), sizeof(int64_t));
    int64_t *nl = malloc(sizeof(int64_t) * (size_t)(cn > 0 ? cn : 1));
    int64_t *lset = malloc(sizeof(int64_t) * (size_t)(cn > 0 ? cn : 1));
    int64_t b[5], tr[3];
    if (!cl || !nl || !lset) { rc = OR_ERR_NOMEM; goto done; }
    for (int64_t t = 1; t <= T && cn > 0; ++t) {
        rc = oracle_run(cn, coff, cadj, variant, 1, p, q, cl, nl, b, lset, tr);   /* one refine iteration */
        if (rc != OR_OK) goto done;
        memcpy(cl, nl, sizeof(int64_t) * (size_t)cn);
        if (trace) { trace[3 * (t - 1)] = b[0]; trace[3 * (t - 1) + 1] = b[1]; trace[3 * (t - 1) + 2] = cn; }
        if (!density_gt(b[0], b[1], se, sv)) continue;                      /* strictly denser? */
        se = b[0]; sv = b[1]; biter = t; ssize = b[3];                       /* S <- S' */
        for (int64_t i = 0; i < ssize; ++i) set[i] = old_of[lset[i]];
        if (density_gt(se, sv, Ln, Ld)) { Ln = se; Ld = sv; }                /* raise L */
        int64_t nlevel = ceil_div(Ln, Ld);
        if (nlevel <= level) continue;
        level = nlevel;                                                      /* re-prune */
        unsigned char *cin = malloc((size_t)cn);
        if (!cin) { rc = OR_ERR_NOMEM; goto done; }
        for (int64_t i = 0; i < cn; ++i) {
            cin[i] = core[old_of[i]] >= level;
            if (!cin[i]) loads[old_of[i]] = cl[i];       /* frozen when pruned */
        }
        int64_t nn = 0, *noff = NULL, *nold = NULL;
        int32_t *nadj = NULL;
        rc = induced_subgraph(cn, coff, cadj, cin, &nn, &noff, &nadj, &nold);
        if (rc != OR_OK) { free(cin); goto done; }
        for (int64_t i = 0; i < nn; ++i) {              /* carry the loads, compose the id maps */
            nl[i] = cl[nold[i]];
            nold[i] = old_of[nold[i]];
        }
        memcpy(cl, nl, sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
        free(cin); free(coff); free(cadj); free(old_of);
        coff = noff; cadj = nadj; old_of = nold; cn = nn;
    }
    for (int64_t i = 0; i < cn; ++i) loads[old_of[i]] = cl[i];
    best[0] = se; best[1] = sv; best[2] = biter; best[3] = ssize; best[4] = 0;
    if (info) { info[3] = cn; info[4] = Ln; info[5] = Ld; }
done:
    free(core); free(in); free(coff); free(cadj); free(old_of); free(cl); free(nl); free(lset);
    return rc;
}

int oracle_run_pruned(int64_t n, const int64_t *off, const int32_t *adj, int variant, int64_t T,
                      int64_t p, int64_t q, int64_t *loads, int64_t *best, int64_t *set, int64_t *trace,
                      int64_t *info)
{
    return oracle_run_pruned_c(n, off, adj, variant, T, p, q, 0, 1, loads, best, set, trace, info);
}

/* PaRApxGreedy++'s pruning (Sec. 4, the approximate variants: approximate
 * k-core pruning followed by exact k-core pruning), read as: the
 * c-approximate decomposition first prunes G to
 * G1 = {v : k-hat(v) >= ceil(k-hat_max / (2c))} (the corollary on the
 * approximate k_max: this bound is at most rho*, so G1 holds S*); then Alg. 1
 * runs with exact pruning on G1 -- the exact core numbers of G1, its k_max,
 * L = ceil(k_max / 2), the L-core of G1 and the refine loop with re-pruning
 * by those core numbers.  Outputs as oracle_run_pruned_c, in the ids of G
 * (vertices outside G1 keep load 0); info[6..8] = (k-hat_max, |V(G1)|,
 * |E(G1)|).                                                                 */
int oracle_run_pruned_ax(int64_t n, const int64_t *off, const int32_t *adj, int variant, int64_t T,
                         int64_t p, int64_t q, int64_t c_num, int64_t c_den, int64_t *loads, int64_t *best,
                         int64_t *set, int64_t *trace, int64_t *info)
{
    if (n < 1 || c_den < 1 || c_num <= c_den) return OR_ERR_INVALID;
    int64_t *khat = malloc(sizeof(int64_t) * (size_t)n);
    unsigned char *in = malloc((size_t)n);
    if (!khat || !in) { free(khat); free(in); return OR_ERR_NOMEM; }
    int rc = oracle_apx_coreness(n, off, adj, c_num, c_den, khat);
    if (rc != OR_OK) { free(khat); free(in); return rc; }
    int64_t khat_max = 0;
    for (int64_t v = 0; v < n; ++v) if (khat[v] > khat_max) khat_max = khat[v];
    const int64_t La = ceil_div(khat_max * c_den, 2 * c_num);      /* approximate stage */
    for (int64_t v = 0; v < n; ++v) in[v] = khat[v] >= La;
    int64_t n1 = 0, *off1 = NULL, *old_of = NULL;
    int32_t *adj1 = NULL;
    rc = induced_subgraph(n, off, adj, in, &n1, &off1, &adj1, &old_of);
    free(khat); free(in);
    if (rc != OR_OK) return rc;
    int64_t *l1 = malloc(sizeof(int64_t) * (size_t)n1);
    int64_t *s1 = malloc(sizeof(int64_t) * (size_t)n1);
    if (!l1 || !s1) { rc = OR_ERR_NOMEM; goto out; }
    rc = oracle_run_pruned_c(n1, off1, adj1, variant, T, p, q, 0, 1, l1, best, s1, trace, info);  /* exact stage */
    if (rc != OR_OK) goto out;
    for (int64_t v = 0; v < n; ++v) loads[v] = 0;
    for (int64_t i = 0; i < n1; ++i) loads[old_of[i]] = l1[i];
    for (int64_t i = 0; i < best[3]; ++i) set[i] = old_of[s1[i]];   /* ascending: old_of is increasing */
    if (info) { info[6] = khat_max; info[7] = n1; info[8] = off1[n1] / 2; }
out:
    free(off1); free(adj1); free(old_of); free(l1); free(s1);
    return rc;
}
