// k_noalloc.cu -- dsg_densest_suffix_noalloc: the densest suffix of the
// (load, id) order for caller-provided device arrays, with every piece of
// scratch memory in one file-scope static device array, so that the call
// allocates nothing.  It drives the same radix-pass kernel (with the fused
// suffix scan) as dsg_run, on scratch carved out of that array.
#include <atomic>
#include <mutex>
#include "common.cuh"
#include "dsg.h"

namespace dsg {
namespace {

constexpr int64_t kNaMaxN = DSG_NOALLOC_MAX_VERTICES;
constexpr int64_t kNaTiles = pass_tiles_max(kNaMaxN);
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffKV = 0;                                        // keys[2], vals[2]
constexpr size_t kOffStatus = kOffKV + al256(16 * (size_t)kNaMaxN);
constexpr size_t kOffStatusSum = kOffStatus + al256(8 * (size_t)kNaTiles * kBuckets);
constexpr size_t kOffCand = kOffStatusSum + al256(16 * (size_t)kNaTiles * kBuckets);
constexpr size_t kOffCtl = kOffCand + al256(sizeof(Candidate) * (size_t)kNaTiles);
constexpr size_t kOffTrace = kOffCtl + al256(sizeof(Control));
constexpr size_t kNaBytes = kOffTrace + al256(3 * sizeof(int64_t));

// All scratch of every call, on every device that loads the library.  Calls
// share it: work that overlaps on the GPU (another stream, another thread)
// races on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
// device address of the array per device, looked up once (under the mutex)
static std::atomic<unsigned char *> g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// The look-back status words and value sums of this call's tiles start at
// zero (flag 0: not published), so a word left behind by an earlier call
// can never be taken for one of this call's, whatever its epoch.
__global__ void k_na_clear(unsigned long long *status, unsigned long long *status_sum, int64_t words)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        status[i] = 0ull;
        status_sum[2 * i] = 0ull;
        status_sum[2 * i + 1] = 0ull;
    }
}

__global__ void k_na_reset(Control *ctl)
{
    ctl->best_e = 0;     // any suffix with an edge is strictly denser than 0/1
    ctl->best_v = 1;
    ctl->best_pos = 0;
    ctl->best_key = 0;
    ctl->best_iter = 0;
    ctl->improved = 0;
    ctl->err = 0;
    ctl->err_where = 0;
    ctl->spin_limit = 0;
    ctl->debug_stall = 0;
    ctl->mm_min[1] = 0xffffffffu;
    ctl->mm_max[1] = 0;
}

__global__ void k_na_minmax(const uint32_t *__restrict__ loads, int64_t n, Control *ctl)
{
    uint32_t mn = 0xffffffffu, mx = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        mn = min(mn, loads[v]);
        mx = max(mx, loads[v]);
    }
    mn = __reduce_min_sync(kFull, mn);
    mx = __reduce_max_sync(kFull, mx);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ctl->mm_min[1], mn);
        atomicMax(&ctl->mm_max[1], mx);
    }
}

// digit counts of (l - lmin) for every pass and per-digit sums of A for the
// last pass (what the edge scan accumulates on the dsg_run path)
__global__ void k_na_hist(const uint32_t *__restrict__ loads, const uint32_t *__restrict__ A,
                          int64_t n, Control *ctl)
{
    __shared__ uint32_t h[kMaxPasses][kBuckets];
    __shared__ unsigned long long as[kBuckets];
    const int np = ctl->npass;
    const uint32_t lmin = ctl->lmin;
    for (int i = threadIdx.x; i < kMaxPasses * kBuckets; i += blockDim.x) (&h[0][0])[i] = 0;
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) as[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = loads[v] - lmin;
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

__global__ void k_na_out(const Control *ctl, const int64_t *trace, int64_t *result)
{
    result[0] = trace[0];
    result[1] = trace[1];
    result[2] = ctl->improved ? ctl->best_pos : 0;
    result[3] = ctl->improved ? ctl->best_key : (int64_t)ctl->lmin;
    result[4] = ctl->err;
}

}  // namespace
}  // namespace dsg

using namespace dsg;

extern "C" int dsg_densest_suffix_noalloc(const uint32_t *loads, const uint32_t *A, int64_t n,
                                          int64_t m, int64_t *result, void *cuda_stream)
{
    // m < 2^48: the last radix pass carries prefix sums in 48-bit tagged words
    if (n < 1 || n > kNaMaxN || m < 0 || (m >> 48) || !loads || !A || !result) return DSG_ERR_INVALID;
    // an error already pending on this thread belongs to someone else: leave
    // it in place and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return DSG_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DSG_ERR_CUDA;
    unsigned char *base = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!base) {
        // once per device, with that device current
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        base = g_scratch_ptr[dev].load(std::memory_order_relaxed);
        if (!base) {
            unsigned char *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();   // this call's own failure
                return DSG_ERR_CUDA;
            }
            g_scratch_ptr[dev].store(p, std::memory_order_release);
            base = p;
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    RunBufs b{};
    uint32_t *kv = (uint32_t *)(base + kOffKV);
    b.keys[0] = kv;
    b.keys[1] = kv + n;
    b.vals[0] = kv + 2 * n;
    b.vals[1] = kv + 3 * n;
    b.loads = const_cast<uint32_t *>(loads);   // read only: the passes run without the load update
    b.A = const_cast<uint32_t *>(A);
    b.status = (unsigned long long *)(base + kOffStatus);
    b.status_sum = (unsigned long long *)(base + kOffStatusSum);
    b.cand = (Candidate *)(base + kOffCand);
    b.ctl = (Control *)(base + kOffCtl);
    b.trace = (int64_t *)(base + kOffTrace);
    b.ntiles = pass_tiles_last(n);
    GraphDev g{};
    g.n = n;
    g.arcs = 2 * m;
    const int grid = (int)imin64((n + 255) / 256, 1024);
    const int64_t words = pass_tiles_max(n) * kBuckets;
    k_na_clear<<<(int)imin64((words + 255) / 256, 1024), 256, 0, s>>>(b.status, b.status_sum, words);
    k_na_reset<<<1, 1, 0, s>>>(b.ctl);
    k_na_minmax<<<grid, 256, 0, s>>>(loads, n, b.ctl);
    if (launch_plan(g, b, 1, s) != cudaSuccess) return DSG_ERR_CUDA;
    k_na_hist<<<grid, 256, 0, s>>>(loads, A, n, b.ctl);
    if (launch_radix_passes(g, b, 1, s, loads, false) != cudaSuccess) return DSG_ERR_CUDA;
    k_na_out<<<1, 1, 0, s>>>(b.ctl, b.trace, result);
    return cudaGetLastError() == cudaSuccess ? DSG_OK : DSG_ERR_CUDA;
}
