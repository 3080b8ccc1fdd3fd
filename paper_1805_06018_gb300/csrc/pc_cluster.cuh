// Thread-block cluster helpers for sm_103a (inline PTX): rank queries, the
// cluster-wide barrier and loads from another CTA's shared memory.
#pragma once

#include <cstdint>

#include "pc_ptx.cuh"

namespace pc {

// ---- thread-block clusters
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// All threads of every CTA of the cluster: memory accesses before the call
// (shared, global) are visible to every thread of the cluster after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 64-bit load from the shared memory of CTA `rank` of the cluster, at the
// address that `local` has in this CTA's shared memory
__device__ __forceinline__ int64_t ld_cluster_s64(const void *local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
    int64_t v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(remote) : "memory");
    return v;
}

}  // namespace pc
