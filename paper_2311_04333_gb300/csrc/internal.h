// internal.h -- layouts shared by the host orchestration (api.cu) and the
// kernels of libdsg.  Not part of the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace dsg {

// ---- edge-scan schedule -----------------------------------------------------
// Vertices of degree > kHeavyDeg are split into chunks of kChunk arcs, one
// work item each (built at upload); all other vertices are taken in groups
// of 32 consecutive ids by single warps, without a list.
// Tuning knobs (compile-time; the defaults are the measured best on GB300).
#ifndef DSG_HUBS
#define DSG_HUBS 12288
#endif
#ifndef DSG_ES_UNROLL
#define DSG_ES_UNROLL 8
#endif
#ifndef DSG_MID_DEG
#define DSG_MID_DEG 64
#endif
#ifndef DSG_ES_THREADS
#define DSG_ES_THREADS 1024
#endif
constexpr int64_t kHeavyDeg = 1024;
constexpr int kChunk = 1024;
// degree orientation: at most kHubs largest-degree vertices get a hub slot;
// oriented arc targets that are hubs are stored as kHubBit | slot
constexpr int kHubs = DSG_HUBS;
constexpr uint32_t kHubBit = 0x80000000u;
// the next tier: at most kHot largest-degree vertices (hubs included) get a
// slot in a dense copy of their loads that stays resident in L2; targets
// outside the hubs but inside it are stored as kHotBit | slot (only when
// n < 2^30, so that plain ids never carry the bit)
#ifndef DSG_HOT
#define DSG_HOT (1 << 23)
#endif
constexpr int64_t kHot = DSG_HOT;
constexpr uint32_t kHotBit = 0x40000000u;
constexpr uint32_t kSlotMask = 0x3fffffffu;

struct WorkItem {
    int64_t a0;      // first arc of the chunk
    uint32_t u;      // the heavy vertex
    uint32_t info;   // its heavy index (accumulator slot)
};

// ---- radix passes -----------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kBuckets = 1 << kRadixBits;
constexpr int kMaxPasses = 4;          // 32-bit keys
constexpr int kPassThreads = 256;      // == kBuckets (one lookback lane per bucket)
#ifndef DSG_PASS_IPT
#define DSG_PASS_IPT 24
#endif
constexpr int kPassIpt = DSG_PASS_IPT;  // items per thread of the last pass
constexpr int kPassTile = kPassThreads * kPassIpt;
#ifndef DSG_PASS_IPT_SCATTER
#define DSG_PASS_IPT_SCATTER 24
#endif
constexpr int kPassIptS = DSG_PASS_IPT_SCATTER;   // items per thread of the scatter passes
constexpr int kPassTileS = kPassThreads * kPassIptS;
// tiles of the last pass, and of whichever pass has more (the look-back
// status words are indexed by tile)
__host__ __device__ constexpr int64_t pass_tiles_last(int64_t n) { return (n + kPassTile - 1) / kPassTile; }
__host__ __device__ constexpr int64_t pass_tiles_scatter(int64_t n) { return (n + kPassTileS - 1) / kPassTileS; }
__host__ __device__ constexpr int64_t pass_tiles_max(int64_t n)
{
    return pass_tiles_last(n) > pass_tiles_scatter(n) ? pass_tiles_last(n) : pass_tiles_scatter(n);
}

// status word of the decoupled look-back: [epoch:16][flag:2][count:46]
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2, kFlagAbort = 3;

// candidate densest suffix of one tile: density edges/vertices, position of
// the suffix's first vertex in the order, and its load key.
struct Candidate {
    int64_t e;
    int64_t v;
    int64_t pos;
    int64_t key;
};

// Per-run control block in device memory.
struct Control {
    // best so far (Alg. 2: S <- G, replaced only on a strictly higher density)
    int64_t best_e, best_v, best_pos;
    int64_t best_key;        // load (at the start of best_iter) of the suffix's first vertex
    int32_t best_iter;
    int32_t improved;        // set by the last pass when this iteration beat the best
    int32_t err;             // dsg_status of a device-side failure (0 = none)
    int32_t err_where;
    // test-only knobs of the bounded waits (dsg_debug_set): polls before a
    // wait gives up (0: kSpinLimit), and a wait made to run out on purpose
    // (1: tile 0 of every radix pass never publishes its look-back words;
    // 2: block 1 never arrives at the first PaRGreedy++ grid barrier)
    uint32_t spin_limit;
    int32_t debug_stall;
    // per-iteration plan (written by the plan kernel)
    uint32_t lmin;           // minimum load at the start of the iteration
    uint32_t lrange;         // max - min load at the start of the iteration
    int32_t npass;           // number of radix passes (>= 1)
    int32_t shift[kMaxPasses];
    uint32_t epoch;          // look-back epoch of pass 0 of this iteration
    // min/max of the next iteration's loads, double-buffered by iteration parity
    uint32_t mm_min[2], mm_max[2];
    // counters
    uint32_t item_ctr;       // edge-scan work-item dispenser
    uint32_t tile_ctr[kMaxPasses];
    uint32_t done_ctr;       // last-tile detection of the final pass
    uint32_t width;          // max deg* of the iteration (empirical width)
    // histograms of the iteration (written by the edge scan)
    uint32_t hist[kMaxPasses][kBuckets];    // counts per digit of (l - lmin)
    unsigned long long asum[kBuckets];       // sum of deg* per digit of the last pass
    // PaRGreedy++ telemetry of the run: rounds, and alive vertices summed over rounds
    unsigned long long peel_rounds, peel_work;
    // best-set materialisation
    int64_t thr_id;          // id of the best suffix's first vertex
    int64_t cnt_less;        // #{v : L(v) < best_key}
    int64_t set_size;
};

// err, err_where, spin_limit and debug_stall are reset together (16 bytes)
// by the runs that do not re-initialise the whole control block
static_assert(offsetof(Control, debug_stall) == offsetof(Control, err) + 12, "Control layout");

// ---- host launchers (implemented in kernels_*.cu) --------------------------
struct GraphDev {
    int64_t n, arcs;         // arcs = 2m
    int64_t max_degree;
    const int64_t *off;
    const int32_t *adj;
    const WorkItem *items;
    int64_t n_items;
    int64_t n_heavy;
    uint32_t *heavy_acc;     // [n_heavy]
    uint32_t *heavy_done;    // [n_heavy]
    // degree-oriented copy used by the sorting edge scan
    const int64_t *ooff;     // [n + 1]
    const uint32_t *oadj;    // [m], targets (hub targets encoded)
    const uint32_t *hub_id;  // [n_hub]
    int64_t n_hub;
    const uint32_t *hot_id;  // [n_hot]
    int64_t n_hot;
    int sorted;              // every adjacency list is strictly ascending
};

struct RunBufs {
    uint32_t *loads;         // l_t (overwritten by l_{t+1} in pass 0)
    uint32_t *A;             // deg* by vertex id
    uint32_t *keys[2];
    uint32_t *vals[2];
    uint32_t *best_loads;    // l_{t*} snapshot of the best iteration
    unsigned long long *status;      // [ntiles * kBuckets]
    unsigned long long *status_sum;  // [ntiles * kBuckets]
    Candidate *cand;         // [ntiles]
    int64_t ntiles;
    Control *ctl;
    int64_t *trace;          // [T * 3] device
    int64_t *blk_a, *blk_b;  // scratch for block-level counts (size nblk64)
    uint32_t *hot_l;         // [n_hot] loads of the hot tier (refreshed per iteration)
    uint32_t *hot_c;         // [n_hot] counts for the hot tier (zero between scans)
    int64_t nblk64;
    void *scratch;           // >= 8n bytes (output staging)
    uint32_t spin_limit = 0; // test-only knobs copied into Control at init
    int32_t debug_stall = 0;
};

// ---- test-only fault hooks (dsg_debug_set, or DSG_FAULT in the environment)
// Process-wide countdowns, off (0) unless a test sets them: when the
// allocation countdown reaches zero, that device (or host context)
// allocation fails as if memory were exhausted; when the upload countdown
// reaches zero, that host-to-device copy of an upload call fails.
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t dev_malloc(T **p, size_t bytes, cudaStream_t s) { return dev_malloc((void **)p, bytes, s); }

// The device buffers one host function allocates on a stream: each is freed
// (stream-ordered, after the work already queued on that stream) when the
// holder goes out of scope, unless handed to the caller with keep().  Every
// return path, including an allocation that fails halfway, so frees what
// the function took and did not hand over.
class DevAllocs {
public:
    explicit DevAllocs(cudaStream_t s) : s_(s) {}
    DevAllocs(const DevAllocs &) = delete;
    DevAllocs &operator=(const DevAllocs &) = delete;
    ~DevAllocs()
    {
        for (int i = 0; i < k_; ++i)
            if (p_[i]) cudaFreeAsync(p_[i], s_);
    }
    template <class T>
    cudaError_t get(T **out, size_t bytes)
    {
        *out = nullptr;
        if (k_ == kMax) return cudaErrorInvalidValue;   // more buffers than one holder tracks
        void *q = nullptr;
        const cudaError_t e = dev_malloc(&q, bytes, s_);
        if (e != cudaSuccess) return e;
        p_[k_++] = q;
        *out = static_cast<T *>(q);
        return cudaSuccess;
    }
    void keep(const void *q)
    {
        for (int i = 0; i < k_; ++i)
            if (p_[i] == q) p_[i] = nullptr;
    }
    void release(void *q)
    {
        for (int i = 0; i < k_; ++i)
            if (p_[i] == q) {
                cudaFreeAsync(q, s_);
                p_[i] = nullptr;
            }
    }

private:
    static constexpr int kMax = 32;
    cudaStream_t s_;
    void *p_[kMax] = {};
    int k_ = 0;
};

bool host_alloc_fault();
bool upload_fault();
void set_alloc_fault(int64_t nth);
void set_upload_fault(int64_t nth);
// bounded waits: polls before a device-side wait gives up (with back-off of
// up to 256 ns per poll this is on the order of a second); a run's Control
// may carry a smaller limit (ctl->spin_limit, test-only)
constexpr uint32_t kSpinLimit = 1u << 22;
__host__ __device__ inline uint32_t spin_limit_of(uint32_t v) { return v ? v : kSpinLimit; }

int edge_scan_sm_count();
// "Compact" graphs (up to 32,768 vertices and 2^20 arcs): their upload
// skips the whole-GPU structures until a whole-GPU run asks for them, and
// the server runs them through the batched kernel, where one block per graph
// is the most work per SM.
constexpr int64_t kCompactN = 1 << 15;
constexpr int64_t kCompactArcs = 1 << 20;
inline bool is_compact(int64_t n, int64_t arcs) { return n <= kCompactN && arcs <= kCompactArcs; }
// Default execution path of dsg_run.  Up to these sizes one thread block
// carrying all T iterations (the kernel of the batched form, on one graph)
// beats the whole-GPU kernels, whose cost there is launches, per-tile
// latency and grid-wide barriers: 16,384 vertices for both variants, with
// 2^18 arcs for PaRSorting++ and 2^19 for PaRGreedy++.
constexpr int64_t kBlockN = 1 << 14;
constexpr int64_t kBlockSortArcs = 1 << 18;
constexpr int64_t kBlockPeelArcs = 1 << 19;
// whole-GPU PaRSorting++ runs up to this many arcs are launched as one CUDA graph
constexpr int64_t kGraphArcs = 1ll << 26;
inline bool block_path_default(int variant, int64_t n, int64_t arcs)
{
    return n <= kBlockN && arcs <= (variant == 1 ? kBlockPeelArcs : kBlockSortArcs);
}

// exclusive scan of int64[count] in place (tmp: scan_tmp_count(count)
// int64 of scratch); *total_dev receives the sum
int64_t scan_tmp_count(int64_t count);
cudaError_t scan_exclusive_i64(int64_t *x, int64_t count, int64_t *total_dev, int64_t *tmp, cudaStream_t s);

cudaError_t launch_validate(const GraphDev &g, int full, int32_t *err_flags, cudaStream_t s);
// err[1..5] of the adjacency alone (as the orientation pass records them)
cudaError_t launch_validate_adjacency(const GraphDev &g, int full, int32_t *err_flags, cudaStream_t s);
int64_t schedule_tmp_count(int64_t n);
cudaError_t build_schedule(GraphDev &g, void *tmp, size_t tmp_bytes, cudaStream_t s,
                           int64_t *n_items_out, int64_t *n_heavy_out, WorkItem **items_out,
                           uint32_t **heavy_mem_out);
cudaError_t launch_init(const GraphDev &g, RunBufs &b, const int64_t *init_dev, int init_is_u32,
                        cudaStream_t s);
cudaError_t launch_plan(const GraphDev &g, RunBufs &b, int t, cudaStream_t s);
cudaError_t launch_edge_scan(const GraphDev &g, RunBufs &b, int grid, cudaStream_t s);
// the passes of the radix sort of (key, A) for the plan of iteration t: the
// scatter passes, then the last pass (which evaluates every suffix); pass 0
// reads key0 (default: the loads) and, if update_loads, writes loads += A.
// accumulate: pass 0 also reduces the width (max A) and, when it is not the
// last pass, the per-digit sums of A for the last pass.  kMaxPasses launches.
// inputs and ping-pong buffers of the passes
struct PassIo {
    const uint32_t *key0, *val0;
    uint32_t *keys0, *keys1, *vals0, *vals1;
};
// one-time kernel attributes of the radix pass (call before any capture)
void radix_prepare();
cudaError_t launch_radix_passes(const GraphDev &g, RunBufs &b, int t, cudaStream_t s,
                                const uint32_t *key0 = nullptr, bool update_loads = true,
                                bool accumulate = false);
cudaError_t launch_snapshot(const GraphDev &g, RunBufs &b, cudaStream_t s);
cudaError_t launch_best_set(const GraphDev &g, RunBufs &b, int32_t *set_dev, cudaStream_t s,
                            int *launches);
cudaError_t launch_loads_out(const GraphDev &g, RunBufs &b, int64_t *dst, cudaStream_t s);
// An adjacency that is still arriving from the host: chunk i holds the
// lists of vertices [v[i], v[i+1]) and is in place once ev[i] has fired.
constexpr int kUploadChunks = 8;
#ifndef DSG_CHUNKED_UPLOAD_ARCS
#define DSG_CHUNKED_UPLOAD_ARCS (1ll << 24)
#endif
constexpr int64_t kChunkedUploadArcs = DSG_CHUNKED_UPLOAD_ARCS;   // smaller host graphs: one copy
struct UploadChunks {
    int k = 0;                          // 0: the whole adjacency is in place
    int64_t v[kUploadChunks + 1] = {};
    cudaEvent_t ev[kUploadChunks] = {};
};
// Validates the adjacency (err[1..5] as in launch_validate; full = symmetry
// and strict order too) while counting the degree-oriented out-degrees, then
// builds the oriented copy unless an error was found.  With chunks, the work
// that needs only the offsets runs while the adjacency arrives, and each
// chunk's counts start as soon as it is in place (all chunks first when
// full: the symmetry check reads other lists).  Returns the number of
// kernel launches in *launches.
cudaError_t build_orientation(GraphDev &g, cudaStream_t s, int full, int32_t *err, int *sorted_out,
                              int64_t **ooff_out, uint32_t **oadj_out, uint32_t **hub_out,
                              int64_t *n_hub_out, uint32_t **hot_out, int64_t *n_hot_out,
                              const UploadChunks *chunks, int *launches);
// copy of bytes (a multiple of 4, 4-byte aligned) from pinned host memory,
// given by its device view, to device memory, by the SMs
cudaError_t launch_copy_h2d(const void *src_dev_view, void *dst, size_t bytes, int sm_count, cudaStream_t s);
cudaError_t launch_asum_single_pass(const GraphDev &g, RunBufs &b, cudaStream_t s);
cudaError_t launch_max_u64_of_i64(const int64_t *src, int64_t n, unsigned long long *dst,
                                  int *neg_flag, cudaStream_t s);
cudaError_t launch_degree_max(const int64_t *off, int64_t n, unsigned long long *dst, cudaStream_t s);

}  // namespace dsg
