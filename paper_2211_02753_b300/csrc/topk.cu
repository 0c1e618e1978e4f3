// K8: ORDER BY value DESC, key ASC LIMIT k (k <= 16).
//
// Each warp keeps one sorted list of its 16 best (value, key) pairs spread
// over lanes 0..15 (lane i holds the i-th best).  The warp reads 32 elements
// at a time; an element is compared with the list's 16th entry (broadcast)
// and almost always rejected there.  The few that qualify are inserted one at
// a time: every lane compares the candidate with its own entry, the ballot
// gives the insertion position, and entries behind it shift down one lane.
// The 8 warp lists of a block are merged the same way by warp 0 and written
// out; a single block then merges the per-block lists.  Lists hold k entries.
// A shared lower bound prunes almost every element before it reaches a
// list: each warp's k-th best so far is at most the global k-th best (its
// elements are a subset), so the running maximum of those values, kept in
// one 64-bit word in the workspace (atomicMax on an order-preserving
// encoding), only ever rejects values that cannot be among the global top
// k; ties at the bound are kept.

#include "topk.cuh"

namespace tdp {

// Pass 1: each lane loads TK_UNROLL values (32 apart) before offering any,
// and the key of a value only when it can enter the list (a key is needed to
// break a tie with the list's last entry or to insert).
constexpr int TK_UNROLL = 8;

__global__ void __launch_bounds__(TK_THREADS) topk_pass1_kernel(const long long *__restrict__ vals,
                                                                const int32_t *__restrict__ keys, long long n_max,
                                                                const long long *d_n, int k, VK *cand,
                                                                unsigned long long *bound)
{
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    WarpList l;
    wl_init(l);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * TK_THREADS * TK_UNROLL;
    long long published = VK_WORST_V;
    // the list's k-th entry, re-read only when an insert changed the list
    long long tv = __shfl_sync(0xffffffffu, l.v, k - 1);
    int tk = __shfl_sync(0xffffffffu, l.k, k - 1);
    for (long long base = ((long long)blockIdx.x * (TK_THREADS / 32) + warp) * 32 * TK_UNROLL; base < n;
         base += stride) {
        long long v[TK_UNROLL];
#pragma unroll
        for (int u = 0; u < TK_UNROLL; u++) {
            const long long i = base + u * 32 + lane;
            v[u] = i < n ? __ldg(vals + i) : VK_WORST_V;
        }
        // the shared bound (relaxed: any value it ever held is a valid bound)
        const long long gb = dec_v(__shfl_sync(0xffffffffu, lane == 0 ? ld_relaxed_u64(bound) : 0ull, 0));
#pragma unroll
        for (int u = 0; u < TK_UNROLL; u++) {
            const long long i = base + u * 32 + lane;
            const bool maybe = i < n && v[u] >= gb && v[u] >= tv;
            const int kk = maybe ? __ldg(keys + i) : VK_WORST_K;
            const unsigned m = __ballot_sync(0xffffffffu, maybe && better(v[u], kk, tv, tk));
            if (m) {
                wl_insert(l, m, v[u], kk, k);
                tv = __shfl_sync(0xffffffffu, l.v, k - 1);
                tk = __shfl_sync(0xffffffffu, l.k, k - 1);
            }
        }
        // publish this warp's k-th best once its list is full and it has risen
        if (tk != VK_WORST_K && tv > published && tv > gb) {
            if (lane == 0)
                atomicMax(bound, enc_v(tv));
            published = tv;
        }
    }
    block_merge(l, k, cand + (size_t)blockIdx.x * k);
}

__global__ void __launch_bounds__(TK_THREADS) topk_pass2_kernel(const VK *__restrict__ cand, long long ncand,
                                                                long long n_max, const long long *d_n, int k,
                                                                long long *out_vals, int32_t *out_keys, long long *d_k,
                                                                const unsigned long long *bound)
{
    const long long gb = dec_v(*bound); // final: every pass-1 block has finished
    __shared__ VK s_out[TK_MAXK];
    WarpList l;
    wl_init(l);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int U = 4; // candidates per lane in flight
    for (long long base = (long long)warp * 32 * U; base < ncand; base += TK_THREADS * U) {
        VK c[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = base + u * 32 + lane;
            c[u] = i < ncand ? cand[i] : VK{VK_WORST_V, VK_WORST_K};
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            wl_offer(l, base + u * 32 + lane < ncand && c[u].v >= gb, c[u].v, c[u].k, k);
    }
    block_merge(l, k, s_out);
    __syncthreads();
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    const long long m = min((long long)k, n);
    if (threadIdx.x < m) {
        out_vals[threadIdx.x] = s_out[threadIdx.x].v;
        out_keys[threadIdx.x] = s_out[threadIdx.x].k;
    }
    if (threadIdx.x == 0 && d_k)
        *d_k = m;
}

static int topk_blocks(long long n)
{
    long long want = (n + TK_THREADS * 32 - 1) / (TK_THREADS * 32);
    return (int)std::max(1ll, std::min<long long>(want, (long long)num_sms() * 2));
}

tdp_status topk_merge(const VK *cand, long long ncand, long long n_max, const long long *d_n, int k,
                      int64_t *out_vals, int32_t *out_keys, int64_t *d_k, const unsigned long long *bound,
                      cudaStream_t s)
{
    topk_pass2_kernel<<<1, TK_THREADS, 0, s>>>(cand, ncand, n_max, d_n, k, (long long *)out_vals, out_keys,
                                               (long long *)d_k, bound);
    return launch_status();
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_topk_workspace(int64_t n, int32_t k)
{
    if (k < 1 || k > TK_MAXK)
        return 0;
    return 256 + align_up((size_t)topk_blocks(n) * k * sizeof(VK), 256); // the bound word, then candidates
}

extern "C" tdp_status tdp_topk(const int64_t *vals, const int32_t *keys, int64_t n, const int64_t *d_n, int32_t k,
                               int64_t *out_vals, int32_t *out_keys, int64_t *d_k, void *ws, size_t ws_bytes,
                               int32_t *d_status, tdp_stream_t stream)
{
    (void)d_status;
    if (n < 0 || k < 1 || k > TK_MAXK || !out_vals || !out_keys || (n > 0 && (!vals || !keys)))
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_topk_workspace(n, k))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    int blocks = topk_blocks(n);
    unsigned long long *bound = (unsigned long long *)ws; // 0 encodes the smallest value: no pruning yet
    VK *cand = (VK *)((char *)ws + 256);
    if (cudaMemsetAsync(bound, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return TDP_ERR_CUDA;
    topk_pass1_kernel<<<blocks, TK_THREADS, 0, s>>>((const long long *)vals, keys, n, (const long long *)d_n, k, cand,
                                                    bound);
    topk_pass2_kernel<<<1, TK_THREADS, 0, s>>>(cand, (long long)blocks * k, n, (const long long *)d_n, k,
                                               (long long *)out_vals, out_keys, (long long *)d_k, bound);
    return launch_status();
}
