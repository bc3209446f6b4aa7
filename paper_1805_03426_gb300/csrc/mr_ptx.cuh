// Inline-PTX helpers shared by the TMA-fed fused step kernels (sm_103a):
// mbarriers with bounded waits, 3-D TMA tile loads, cp.async, and a barrier
// among the consumer warps only.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace mr {
namespace ptx {

constexpr long kWaitLimit = 1L << 26;                  // bounded mbarrier wait: iterations ...
constexpr unsigned long long kWaitNs = 1000000000ull;  // ... and wall time (1 s, unless a launch gives less)

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
// Barrier among the consumer warps only (the producer warp never joins).
template <int N>
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("barrier.cta.sync 1, %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ bool consumers_sync_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.cta.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(N)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity), "n"(20000)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait (iteration count and wall time limit_ns); true on success.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, unsigned long long limit_ns = kWaitNs)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long it = 0; it < kWaitLimit; ++it) {
        if (mbar_test(b, parity)) return true;
        if ((it & 15) == 0 && global_ns() - t0 > limit_ns) break;
    }
    return false;
}
// Bounded wait for a warp with slack (a producer that runs ahead of its
// consumers, a builder a slab ahead): between polls it sleeps sleep_ns, so
// that its polling does not take issue slots from the warps on the critical
// path.  true on success.
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* b, uint32_t parity, unsigned long long limit_ns,
                                               unsigned sleep_ns)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long it = 0; it < kWaitLimit; ++it) {
        __nanosleep(sleep_ns);
        if (mbar_test(b, parity)) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    return false;
}
__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(sa(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }


}  // namespace ptx
}  // namespace mr
