// Inline-PTX helpers for sm_103a: mbarriers, bulk (TMA) copies, cp.async,
// acquire/release flags.
#pragma once

#include <cstdint>

namespace pc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of asynchronous transfer
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier: false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Device wall clock in nanoseconds (for waits bounded in time).
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait limit of an apply's device-side waits when the operator sets none: 2 s.
constexpr int64_t kDefaultWaitNs = 2000000000ll;
__device__ __forceinline__ int64_t wait_limit_ns(int64_t ns) { return ns > 0 ? ns : kDefaultWaitNs; }

// Wait for phase `parity` of an mbarrier for at most limit_ns: false if it
// gave up.  Only time bounds it: an asynchronous copy into this CTA's shared
// memory must land before the CTA reuses the buffer or exits.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t *bar, uint32_t parity, int64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (int64_t(global_ns() - t0) > limit_ns) return false;
    }
}

// Bulk global -> shared copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Order this thread's earlier generic-proxy shared accesses before later
// asynchronous-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// release store at system scope (the host reads the word through mapped memory)
__device__ __forceinline__ void st_release_sys_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// acquire load at system scope (a word the host writes in mapped memory)
__device__ __forceinline__ uint32_t ld_acquire_sys_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_volatile_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *f == want (acquire; system scope for a host-written word),
// for at most limit_ns.  The launch's status word makes the waits sticky:
// once any wait of the launch has given up (status != 0) every other wait
// gives up at once, so a failed launch ends within about one limit.  On a
// timeout the first waiter to give up records `code` in the status word.
// Returns true if the flag arrived.
template <bool SYS>
__device__ __forceinline__ bool wait_flag_eq(const uint32_t *f, uint32_t want, int32_t *status, int64_t limit_ns,
                                             int32_t code, unsigned sleep_ns) {
    auto ld = [&]() { return SYS ? ld_acquire_sys_u32(f) : ld_acquire_u32(f); };
    if (ld() == want) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        __nanosleep(sleep_ns);
        if (ld() == want) return true;
        if ((it & 7u) == 0u) {
            if (ld_volatile_s32(status) != 0) return false;
            if (int64_t(global_ns() - t0) > limit_ns) {
                atomicCAS(status, 0, code);
                return false;
            }
        }
    }
}

}  // namespace pc

namespace pc {

// Bulk reduction shared -> global: dst[i] += src[i] (f32) for bytes/4 values,
// performed by the asynchronous (TMA) unit.  16-byte aligned addresses, size a
// multiple of 16.  Tracked by this thread's bulk async-groups.
__device__ __forceinline__ void bulk_reduce_add_f32(float *dst, const float *src, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk groups have finished reading their shared-memory sources
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk groups are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

}  // namespace pc
