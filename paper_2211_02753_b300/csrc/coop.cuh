// Block-level scans and the one-barrier cooperative prefix shared by the
// cooperative passes (group-join rank / hit-rank, N:M join): blocks of
// COOP_THREADS threads.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tdp {

constexpr int COOP_THREADS = 256;

// Exclusive block scan of one unsigned per thread; returns the thread's
// exclusive prefix and (in *total) the block total.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *s_warp, unsigned *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    unsigned before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < COOP_THREADS / 32; w++) {
        const unsigned t = s_warp[w];
        before += w < warp ? t : 0;
        all += t;
    }
    *total = all;
    return before + incl - v;
}

// Block-wide sum of one value per thread (every thread gets the total).
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long *s_red)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads(); // s_red free from an earlier use
    if (lane == 0)
        s_red[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < COOP_THREADS / 32; w++)
        t += s_red[w];
    return t;
}

// Every block of a cooperative launch publishes its total, waits once on a
// bounded grid-wide barrier for all blocks to have counted, and returns the
// sum of the totals of the blocks before it.
__device__ __forceinline__ unsigned long long coop_block_prefix(unsigned long long block_total,
                                                                unsigned long long *s_red,
                                                                unsigned long long *totals, unsigned *barrier,
                                                                uint32_t limit, int32_t *d_status)
{
    if (threadIdx.x == 0)
        st_relaxed_u64(&totals[blockIdx.x], block_total);
    grid_barrier(barrier, gridDim.x, limit, d_status);
    unsigned long long before = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += COOP_THREADS)
        before += ld_relaxed_u64(&totals[b]);
    return block_sum(before, s_red);
}

} // namespace tdp

namespace tdp {

// 64-bit exclusive block scan (same contract as block_excl_scan).
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v, unsigned long long *s_warp,
                                                                unsigned long long *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < COOP_THREADS / 32; w++) {
        const unsigned long long t = s_warp[w];
        before += w < warp ? t : 0;
        all += t;
    }
    *total = all;
    return before + incl - v;
}

// Blocks of a cooperative launch of `kern` (COOP_THREADS threads, no dynamic
// shared memory) covering `units` work units of `per_block` units each: as
// many as are resident at once at most, each taking `rounds` consecutive
// spans.  False if the occupancy query fails.
inline bool coop_grid_for(const void *kern, long long units, long long per_block, int *G, int *rounds)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, COOP_THREADS, 0) != cudaSuccess || per_sm < 1)
        return false;
    const long long spans = std::max(1ll, (units + per_block - 1) / per_block);
    const long long res = (long long)per_sm * num_sms();
    *rounds = (int)((spans + res - 1) / res);
    *G = (int)((spans + *rounds - 1) / *rounds);
    return true;
}

} // namespace tdp

namespace tdp {

// coop_block_prefix for two totals at once (one barrier): totals holds
// 2 x gridDim.x words.
__device__ __forceinline__ void coop_block_prefix2(unsigned long long t0, unsigned long long t1,
                                                   unsigned long long *s_red, unsigned long long *totals,
                                                   unsigned *barrier, uint32_t limit, int32_t *d_status,
                                                   unsigned long long *p0, unsigned long long *p1)
{
    if (threadIdx.x == 0) {
        st_relaxed_u64(&totals[2 * blockIdx.x], t0);
        st_relaxed_u64(&totals[2 * blockIdx.x + 1], t1);
    }
    grid_barrier(barrier, gridDim.x, limit, d_status);
    unsigned long long b0 = 0, b1 = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += COOP_THREADS) {
        b0 += ld_relaxed_u64(&totals[2 * b]);
        b1 += ld_relaxed_u64(&totals[2 * b + 1]);
    }
    *p0 = block_sum(b0, s_red);
    *p1 = block_sum(b1, s_red);
}

} // namespace tdp
