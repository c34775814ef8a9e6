// cbg_tc.cuh -- 5th-generation tensor core (tcgen05) primitives for sm_100-class GPUs, as
// inline PTX: shared-memory operand descriptors, MMA issue and commit, tensor-memory
// allocation and loads, and the fences that order them against ordinary threads.
//
// Operand tiles are K-major with the 128-byte swizzle: row m of a tile is one 128-byte
// line of 64 16-bit K values at m * 128, its 16-byte chunk c stored at chunk position
// c ^ (m & 7), so eight consecutive rows spread one K chunk over all banks.  Tile bases
// are 1024-byte aligned; one MMA consumes K = 16 values, and the next K step starts 32
// bytes further inside the same swizzle atom.
#pragma once
#include <cstdint>

#include "cbg_tma.cuh"

namespace cbg {

constexpr int TC_ROWB = 128;              // bytes of one operand row (64 16-bit K values)
constexpr int TC_SBO = 8 * TC_ROWB;       // bytes between 8-row groups

__host__ __device__ constexpr int tc_swz(int m, int chunk) { return m * TC_ROWB + ((chunk ^ (m & 7)) << 4); }

// shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand starting at addr
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                      // leading offset: unused for swizzled K-major
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// instruction descriptor of kind::f16 with FP32 accumulation, both operands K-major:
// A and B both FP16 (bf16 = false) or both BF16
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, bool bf16)
{
    return (1u << 4) | (bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B^T (+ D when acc != 0), issued by one thread
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive once on bar when every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive tensor-memory columns of this warp's 32 lanes (completed by tc_wait_ld)
__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ordinary shared-memory stores of this thread become visible to the tensor core
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// allocate `cols` tensor-memory columns (a power of two >= 32) for this CTA; executed by
// one whole warp; the base address lands in *dst (shared memory)
__device__ __forceinline__ void tc_alloc(uint32_t* dst, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

}  // namespace cbg
