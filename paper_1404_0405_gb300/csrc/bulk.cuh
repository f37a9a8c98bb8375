// Asynchronous copies from global to shared memory (PTX ISA: cp.async.bulk,
// mbarrier, cp.async).  One-dimensional bulk copies by the tensor memory
// accelerator complete on an mbarrier in shared memory; a bulk copy moves a
// multiple of 16 bytes between 16-byte aligned addresses, and the waits on its
// mbarrier are bounded (a wait that does not see its phase complete within
// `limit` clock cycles returns false).  Element copies (4 or 8 bytes) complete
// per thread.
#pragma once
#include <cstdint>

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// an mbarrier with one arriving thread (the thread that starts the copies); call
// from one thread, then fence_barrier_init and a block barrier before first use
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// makes mbarrier initialisations visible to the copy engine
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// the arriving thread announces `bytes` on bar and starts the copy src -> dst;
// bar's current phase completes when they have landed
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// true once the phase of bar with parity `parity` has completed (its copies are
// visible to the calling thread); false after `limit` cycles without completion
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Element copies from global to shared memory that do not hold the issuing thread
// (cp.async, size 4 or 8 bytes, both addresses aligned to it); a thread's copies
// are grouped by async_commit and waited for by async_wait_all.
template <int BYTES>
__device__ __forceinline__ void async_copy(void* dst, const void* src) {
    static_assert(BYTES == 4 || BYTES == 8, "element copy size");
    if constexpr (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
