// Thread-block cluster primitives (inline PTX for sm_103a): rank queries, the cluster-wide
// barrier with release / acquire semantics, and loads / stores into the shared memory of
// another CTA of the cluster (distributed shared memory, addresses mapped with mapa).
#pragma once
#include <cuda_runtime.h>

namespace hm {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_map(unsigned a, unsigned rank)
{
    unsigned d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
__device__ __forceinline__ unsigned ld_cluster_u32(unsigned a)
{
    unsigned v;
    asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float2 ld_cluster_f2(unsigned a)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ void st_cluster_u32(unsigned a, unsigned v)
{
    asm volatile("st.relaxed.cluster.shared::cta.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// plain stores into the shared memory of a cluster CTA (address from cluster_map); a cluster
// barrier (release / acquire) orders them before the owner's reads
__device__ __forceinline__ void st_remote_d2(unsigned a, double2 v)
{
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void st_remote_s32(unsigned a, int v)
{
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

}  // namespace hm
