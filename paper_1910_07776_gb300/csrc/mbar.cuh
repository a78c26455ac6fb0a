// mbar.cuh -- mbarrier and TMA bulk-copy helpers (inline PTX) shared by the kernels that
// stage global memory through shared memory asynchronously: the tensor-core GEMM core and
// the rank pass.  Every wait is bounded (1 s of %globaltimer); a wait that gives up sets
// RS_ETIMEOUT in the device status word and returns false, and its caller drains its own
// copies in flight (with the same bound) before leaving.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_internal.cuh"

namespace tc {

constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed, false (and RS_ETIMEOUT flagged with the
// caller's site number) after limit_ns of %globaltimer.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t phase, int* err, int site,
                                              unsigned long long limit_ns) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        if (gtime() - t0 > limit_ns) {
            rs_dev_flag(err, RS_ETIMEOUT, site);
            return false;
        }
    }
}
// The kernels' wait: bounded by 1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, int* err, int site) {
    return mbar_wait_for(bar, phase, err, site, kWaitNs);
}
// 1-D bulk copy global -> shared (TMA, non-tensor form), completing on the mbarrier's
// transaction count.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace tc
