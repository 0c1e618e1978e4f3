// cp.async helpers of the glyph-CNN kernels: 16-byte global -> shared copies
// (zero fill when the source is absent) and their commit/wait groups.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace tdp {
namespace cnn {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    const int sz = valid ? 16 : 0; // src-size 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(valid ? gmem : (const void *)0),
                 "r"(sz)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

} // namespace cnn
} // namespace tdp
