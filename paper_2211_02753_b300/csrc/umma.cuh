// 5th-generation tensor core (tcgen05) helpers: tensor-memory allocation,
// shared-memory operand descriptors, the bf16 MMA with fp32 accumulation in
// tensor memory, its commit to an mbarrier, and the accumulator loads.
//
// Operand layout in shared memory (K-major, no swizzle): the operand is cut
// into core matrices of 8 rows x 16 bytes (8 bf16 along K), each stored as
// 128 contiguous bytes (row r of the core matrix at r * 16).  The core
// matrices of one 8-row group that follow each other along K are LBO bytes
// apart, and consecutive 8-row groups SBO bytes apart.  The tiles here put
// the K chunks of a row group next to each other: LBO = 128, SBO = (K of the
// tile / 8) * 128.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace tdp {
namespace umma {

// Shared-memory matrix descriptor: start address, LBO and SBO (all >> 4),
// descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Descriptor of a K-major operand stored with the 128-byte swizzle: each row
// of 64 bf16 (one K stage) is 128 bytes, 8 rows form a 1024-byte atom whose
// 16-byte chunks are XOR-permuted by row (the layout a TMA copy with
// CU_TENSOR_MAP_SWIZZLE_128B writes); SBO = 1024 (the next 8 rows), LBO
// unused (1), layout type 2 (128-byte swizzle) in bits 61-63.  The atom must
// be 1024-byte aligned; a K16 step advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Descriptor of an MN-major operand stored with the 128-byte swizzle: each
// k-row holds 64 consecutive M (or N) elements in 128 bytes, 8 k-rows form a
// 1024-byte atom.  Here the leading offset is the distance between 64-element
// groups along M/N and the stride offset the distance between 8-row groups
// along K (measured: the other assignment gives wrong products); layout type
// 2.
__device__ __forceinline__ uint64_t smem_desc_sw128_mn(uint32_t saddr, uint32_t k_stride, uint32_t mn_stride)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((mn_stride >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((k_stride >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major) and an
// fp32 accumulator: D format bit 4, A format bits 7-9 = 1 (bf16), B format
// bits 10-12 = 1, N / 8 at bit 17, M / 16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocates ncols tensor-memory columns (a power of two >= 32); one full warp
// calls it; the address lands in *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tensor memory) [+]= A * B^T for one K step of 16; issued by one thread.
// True in exactly one lane of a converged warp (elect.sync): the issuing
// lane of a warp that runs the MMA loop with warp-uniform descriptors.
__device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.b32 %0, 1, 0, P;\n\t}"
                 : "=r"(pred));
    return pred != 0;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1 : 0)
                 : "memory");
}

// The mbarrier gets one arrival once every MMA this thread issued so far has
// completed.
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive fp32 columns of the calling thread's tensor-memory lane
// (warp w of a 128-thread group reads lanes 32w..32w+31).
__device__ __forceinline__ void ld_16cols(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++)
        v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk (row r, k chunk kc) in a K-major tile whose
// rows hold KC chunks.
__device__ __forceinline__ uint32_t chunk_off(int r, int kc, int KC)
{
    return (uint32_t)((r >> 3) * (KC * 128) + kc * 128 + (r & 7) * 16);
}

} // namespace umma
} // namespace tdp
