// common.cuh -- small device helpers shared by the kernels of libdsg.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "internal.h"

namespace dsg {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// exact comparison of densities e1/v1 > e2/v2 (v1, v2 > 0), 128-bit products
__device__ __forceinline__ bool dens_gt(uint64_t e1, uint64_t v1, uint64_t e2, uint64_t v2)
{
    uint64_t ah = __umul64hi(e1, v2), al = e1 * v2;
    uint64_t bh = __umul64hi(e2, v1), bl = e2 * v1;
    return ah > bh || (ah == bh && al > bl);
}

// candidate order: higher density first, then the earlier position (the
// larger suffix), i.e. the first maximum of the suffix densities in order.
__device__ __forceinline__ bool cand_better(const Candidate &a, const Candidate &b)
{
    if (a.v <= 0) return false;
    if (b.v <= 0) return true;
    if (dens_gt((uint64_t)a.e, (uint64_t)a.v, (uint64_t)b.e, (uint64_t)b.v)) return true;
    if (dens_gt((uint64_t)b.e, (uint64_t)b.v, (uint64_t)a.e, (uint64_t)a.v)) return false;
    return a.pos < b.pos;
}

__device__ __forceinline__ Candidate shfl_cand(const Candidate &c, int src)
{
    Candidate r;
    r.e = __shfl_sync(kFull, c.e, src);
    r.v = __shfl_sync(kFull, c.v, src);
    r.pos = __shfl_sync(kFull, c.pos, src);
    r.key = __shfl_sync(kFull, c.key, src);
    return r;
}

__device__ __forceinline__ Candidate warp_best(Candidate c)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Candidate x = shfl_cand(c, (threadIdx.x & 31) ^ o);
        if (cand_better(x, c)) c = x;
    }
    return c;
}

// block-wide best candidate (blockDim.x multiple of 32, <= 1024); result
// valid in every thread.  `sm` must hold 32 Candidates.
__device__ __forceinline__ Candidate block_best(Candidate c, Candidate *sm)
{
    c = warp_best(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sm[w] = c;
    __syncthreads();
    Candidate r = (l < nw) ? sm[l] : Candidate{0, 0, 0, 0};
    r = warp_best(r);
    return r;
}

// block-wide exclusive sum over one uint64 per thread; `sm` holds 33 entries.
__device__ __forceinline__ uint64_t block_excl_sum_u64(uint64_t x, unsigned long long *sm, uint64_t *total)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    uint64_t inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, inc, o);
        if (l >= o) inc += y;
    }
    __syncthreads();
    if (l == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint64_t s = (l < nw) ? sm[l] : 0, si = s;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, si, o);
            if (l >= o) si += y;
        }
        if (l < nw) sm[l] = si - s;
        if (l == 31) sm[32] = si;
    }
    __syncthreads();
    uint64_t r = sm[w] + inc - x;
    if (total) *total = sm[32];
    return r;
}

// record a device-side failure (first one wins)
__device__ __forceinline__ void set_error(Control *ctl, int code, int where)
{
    if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_where = where;
}

}  // namespace dsg
