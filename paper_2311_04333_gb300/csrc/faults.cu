// faults.cu -- test-only fault hooks of libdsg (host code).  Failure paths
// are tested by making the failure on the host: an allocation that reports
// exhausted memory, or an upload copy that fails, at a chosen point.  Both
// countdowns are process-wide and off unless dsg_debug_set or the DSG_FAULT
// environment variable ("alloc:N", "upload:N", comma-separated; read when
// the library is loaded) turns them on.
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "internal.h"

namespace dsg {
namespace {

std::atomic<int64_t> g_alloc_countdown{0};
std::atomic<int64_t> g_upload_countdown{0};

// true when this tick takes the countdown from 1 to 0
bool tick(std::atomic<int64_t> &c)
{
    int64_t v = c.load(std::memory_order_relaxed);
    while (v > 0) {
        if (c.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
    }
    return false;
}

struct EnvFaults {
    EnvFaults()
    {
        const char *e = std::getenv("DSG_FAULT");
        if (!e) return;
        const char *p = e;
        while (*p) {
            const char *colon = std::strchr(p, ':');
            if (!colon) break;
            const int64_t nth = std::strtoll(colon + 1, nullptr, 10);
            if (!std::strncmp(p, "alloc", 5)) g_alloc_countdown = nth;
            else if (!std::strncmp(p, "upload", 6)) g_upload_countdown = nth;
            const char *comma = std::strchr(colon, ',');
            if (!comma) break;
            p = comma + 1;
        }
    }
} g_env_faults;

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s)
{
    if (tick(g_alloc_countdown)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

bool host_alloc_fault() { return tick(g_alloc_countdown); }
bool upload_fault() { return tick(g_upload_countdown); }
void set_alloc_fault(int64_t nth) { g_alloc_countdown = nth > 0 ? nth : 0; }
void set_upload_fault(int64_t nth) { g_upload_countdown = nth > 0 ? nth : 0; }

}  // namespace dsg
