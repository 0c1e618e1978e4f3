// Top-k building blocks shared by tdp_topk and the group-join's fused top-k:
// warp-wide sorted lists of (value, key) pairs ordered by value desc, key
// asc, their block merge, and the final single-block merge of per-block
// candidate lists.
#pragma once

#include "common.cuh"

namespace tdp {

constexpr int TK_THREADS = 256;
constexpr int TK_LIST = 16;
constexpr int TK_MAXK = 16;

struct VK {
    long long v;
    int k;
};

__device__ __forceinline__ bool better(long long av, int ak, long long bv, int bk)
{
    return av > bv || (av == bv && ak < bk);
}

constexpr long long VK_WORST_V = (long long)0x8000000000000000ull;
constexpr int VK_WORST_K = 0x7fffffff;

// Warp-wide sorted list: lane i < 16 holds entry i (lanes >= 16 hold copies
// of the worst value and never matter).
struct WarpList {
    long long v;
    int k;
};

__device__ __forceinline__ void wl_init(WarpList &l)
{
    l.v = VK_WORST_V;
    l.k = VK_WORST_K;
}

// Inserts the candidates held by the lanes in `mask` (each lane's (cv, ck))
// into the list of the first k lanes.
__device__ __forceinline__ void wl_insert(WarpList &l, unsigned mask, long long cv, int ck, int k)
{
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const long long xv = __shfl_sync(0xffffffffu, cv, src);
        const int xk = __shfl_sync(0xffffffffu, ck, src);
        // position = number of entries that stay ahead of x
        const unsigned ahead = __ballot_sync(0xffffffffu, lane < k && !better(xv, xk, l.v, l.k));
        const int pos = __popc(ahead);
        if (pos >= k)
            continue;
        const long long uv = __shfl_up_sync(0xffffffffu, l.v, 1);
        const int uk = __shfl_up_sync(0xffffffffu, l.k, 1);
        if (lane == pos) {
            l.v = xv;
            l.k = xk;
        } else if (lane > pos && lane < k) {
            l.v = uv;
            l.k = uk;
        }
    }
}

// Offers one element per lane (valid lanes only) to a k-entry list.
__device__ __forceinline__ void wl_offer(WarpList &l, bool valid, long long v, int key, int k)
{
    const long long tv = __shfl_sync(0xffffffffu, l.v, k - 1);
    const int tk = __shfl_sync(0xffffffffu, l.k, k - 1);
    const unsigned m = __ballot_sync(0xffffffffu, valid && better(v, key, tv, tk));
    if (m)
        wl_insert(l, m, v, key, k);
}

// Order-preserving unsigned encoding of a signed value (for atomicMax).
__device__ __forceinline__ unsigned long long enc_v(long long v)
{
    return (unsigned long long)v ^ 0x8000000000000000ull;
}
__device__ __forceinline__ long long dec_v(unsigned long long e) { return (long long)(e ^ 0x8000000000000000ull); }

// Merges the warp lists of the block; warp 0 writes the first k to out.
__device__ __forceinline__ void block_merge(WarpList &l, int k, VK *out)
{
    __shared__ VK s_c[TK_THREADS / 32 * TK_LIST];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < TK_LIST)
        s_c[warp * TK_LIST + lane] = VK{l.v, l.k};
    __syncthreads();
    if (warp == 0) {
        WarpList m;
        wl_init(m);
        for (int base = 0; base < TK_THREADS / 32 * TK_LIST; base += 32) {
            VK c = s_c[base + lane];
            wl_offer(m, true, c.v, c.k, k);
        }
        if (lane < k)
            out[lane] = VK{m.v, m.k};
    }
}

// Merges `ncand` candidate entries (per-block lists of k entries, missing
// entries holding the worst value) into the first min(k, n) results, n =
// *d_n (or n_max); values below *bound are known not to be among them.
tdp_status topk_merge(const VK *cand, long long ncand, long long n_max, const long long *d_n, int k,
                      int64_t *out_vals, int32_t *out_keys, int64_t *d_k, const unsigned long long *bound,
                      cudaStream_t s);

} // namespace tdp
