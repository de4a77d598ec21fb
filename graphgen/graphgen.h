/*
 * graphgen.h -- seeded synthetic graph recipes shared by the CPU generator
 * (graphgen.c) and the GPU generator (graphgen_cuda.cu).  Holds no part of
 * the densest-subgraph method: only random numbers and graph recipes.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: the i-th draw of stream `key` is mix64(key + (i+1)*GOLDEN),
 * i.e. the (i+1)-th output of a SplitMix64 whose state starts at `key`.
 * A stream key is derived from (seed, stream id) as
 * mix64(seed*GOLDEN ^ mix64(stream + GOLDEN)).
 */
#ifndef GRAPHGEN_H
#define GRAPHGEN_H
#include <stdint.h>

#if defined(__CUDACC__)
#define GG_FN __host__ __device__ __forceinline__
#else
#define GG_FN static inline
#endif

#define GG_GOLDEN 0x9E3779B97F4A7C15ull

GG_FN uint64_t gg_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

GG_FN uint64_t gg_key(uint64_t seed, uint64_t stream)
{
    return gg_mix64(seed * GG_GOLDEN ^ gg_mix64(stream + GG_GOLDEN));
}

GG_FN uint64_t gg_draw(uint64_t key, uint64_t i)
{
    return gg_mix64(key + (i + 1ull) * GG_GOLDEN);
}

/* R-MAT quadrant thresholds in units of 1/65536:
 * a = 0.57 -> 37355, b = c = 0.19 -> 12451, d = the rest (3279/65536). */
#define GG_RMAT_A 37355u
#define GG_RMAT_B 12451u
#define GG_RMAT_C 12451u

/* Stream ids used by the recipes. */
#define GG_STREAM_ER 1ull
#define GG_STREAM_CLIQUE 2ull
#define GG_STREAM_RMAT 3ull
#define GG_STREAM_BLOCK_PERM 4ull
#define GG_STREAM_BLOCK_EDGES 16ull /* + block index */

/* Endpoints of R-MAT edge i at `scale` (Chakrabarti, Zhan and Faloutsos,
 * "R-MAT: A recursive model for graph mining", SDM 2004): `scale` levels,
 * most significant bit first; level L uses the 16-bit chunk L%4 of draw
 * i*ceil(scale/4) + L/4.  Quadrants: (0,0) a, (0,1) b, (1,0) c, (1,1) d. */
GG_FN void gg_rmat_edge(uint64_t key, int scale, uint64_t i, uint32_t *pu, uint32_t *pv)
{
    uint32_t u = 0, v = 0;
    uint64_t per = (uint64_t)((scale + 3) / 4);
    uint64_t r = 0;
    for (int L = 0; L < scale; ++L) {
        if ((L & 3) == 0) r = gg_draw(key, i * per + (uint64_t)(L >> 2));
        uint32_t x = (uint32_t)(r >> (16 * (L & 3))) & 0xFFFFu;
        uint32_t ub, vb;
        if (x < GG_RMAT_A) { ub = 0; vb = 0; }
        else if (x < GG_RMAT_A + GG_RMAT_B) { ub = 0; vb = 1; }
        else if (x < GG_RMAT_A + GG_RMAT_B + GG_RMAT_C) { ub = 1; vb = 0; }
        else { ub = 1; vb = 1; }
        u = (u << 1) | ub;
        v = (v << 1) | vb;
    }
    *pu = u;
    *pv = v;
}

/* Planted dense blocks on an R-MAT id space of 2^scale vertices: block b has
 * s_b vertices perm(base_b + j), j < s_b, where perm(x) = (x*mul + add) mod
 * 2^scale is a bijection (mul odd) and the bases are disjoint ranges, so the
 * blocks are disjoint.  Pair (i < j) of block b is an edge iff draw
 * i*s_b + j of stream GG_STREAM_BLOCK_EDGES + b has its top bit clear
 * (probability 1/2). */
GG_FN uint32_t gg_block_vertex(uint64_t mul, uint64_t add, int scale, uint64_t x)
{
    uint64_t mask = (scale >= 64) ? ~0ull : ((1ull << scale) - 1ull);
    return (uint32_t)((x * mul + add) & mask);
}

#endif
