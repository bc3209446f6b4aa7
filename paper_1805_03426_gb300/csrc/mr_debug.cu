// Test hooks of the failure paths (no counterpart in the paper).  Both make a
// failure on the host side of a call, never a GPU fault:
//   - a one-shot shortened wait limit for the next TMA step launch, whose
//     producer in one CTA stops issuing its ring part-way, so that the
//     consumers' bounded waits run out and the launch reports MR_ERR_TIMEOUT
//     through the device flag (every ring issued before the stop is still
//     waited for, so no copy is left in flight when the CTA exits);
//   - a cap on the library's device allocations, which refuses an allocation
//     the way cudaMalloc does when memory runs out (MR_ERR_OOM), and a count of
//     the bytes held, so that a test can check that a failed call frees what
//     it took.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "mr_internal.cuh"
#include "mr_ptx.cuh"

namespace mr {
namespace {

std::mutex g_inj_mu;
int g_inj_ring = -1;
unsigned long long g_inj_ns = 0;

std::mutex g_mem_mu;
std::unordered_map<void*, size_t> g_live;
long long g_live_bytes = 0;
long long g_cap = -1;   // -1: no cap

}  // namespace

void take_wait_injection(int* stop_ring, unsigned long long* wait_ns)
{
    std::lock_guard<std::mutex> lock(g_inj_mu);
    if (g_inj_ring < 0) return;
    *stop_ring = g_inj_ring;
    *wait_ns = g_inj_ns;
    g_inj_ring = -1;
}

cudaError_t dev_malloc(void** p, size_t bytes)
{
    std::lock_guard<std::mutex> lock(g_mem_mu);
    if (g_cap >= 0 && g_live_bytes + (long long)bytes > g_cap) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    g_live[*p] = bytes;
    g_live_bytes += (long long)bytes;
    return cudaSuccess;
}

cudaError_t dev_free(void* p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_mem_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            g_live_bytes -= (long long)it->second;
            g_live.erase(it);
        }
    }
    return cudaFree(p);
}

}  // namespace mr

using namespace mr;

extern "C" {

int mr_debug_inject_wait_timeout(int32_t stop_ring, double wait_seconds)
{
    if (stop_ring < 0 || !(wait_seconds > 0) || wait_seconds > 1.0)
        return set_error(MR_ERR_ARG, "mr_debug_inject_wait_timeout: stop_ring >= 0 and 0 < wait_seconds <= 1");
    std::lock_guard<std::mutex> lock(g_inj_mu);
    g_inj_ring = stop_ring;
    g_inj_ns = (unsigned long long)(wait_seconds * 1e9);
    return MR_OK;
}

int mr_debug_alloc_cap(int64_t cap_bytes, int64_t* live_bytes)
{
    if (cap_bytes < -2) return set_error(MR_ERR_ARG, "mr_debug_alloc_cap: cap_bytes must be >= -2");
    std::lock_guard<std::mutex> lock(g_mem_mu);
    if (cap_bytes != -2) g_cap = cap_bytes;
    if (live_bytes) *live_bytes = g_live_bytes;
    return MR_OK;
}

}  // extern "C"
