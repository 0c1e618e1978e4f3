// K8: ORDER BY value DESC, key ASC LIMIT k (k <= 16).
//
// Pass 1: every thread keeps the 16 best (value, key) pairs of its strided
// share of the input in a sorted register list (insertions are rare once the
// list is warm: an element is compared with the current 16th best first).
// The block then extracts its k best with k rounds of a block-wide arg-max
// over the threads' list heads; the winner pops its head.  Pass 2: one block
// does the same over the per-block candidates.
#include "common.cuh"

namespace tdp {

constexpr int TK_THREADS = 256;
constexpr int TK_LIST = 16;
constexpr int TK_MAXK = 16;

struct VK {
    long long v;
    int k;
};

__device__ __forceinline__ bool better(const VK &a, const VK &b) { return a.v > b.v || (a.v == b.v && a.k < b.k); }

__device__ __forceinline__ VK worst_vk()
{
    VK w;
    w.v = (long long)0x8000000000000000ull;
    w.k = 0x7fffffff;
    return w;
}

__device__ __forceinline__ void list_insert(VK (&L)[TK_LIST], const VK &x)
{
    if (!better(x, L[TK_LIST - 1]))
        return;
    bool placed = false;
#pragma unroll
    for (int i = TK_LIST - 1; i >= 1; i--) {
        if (!placed) {
            if (better(x, L[i - 1])) {
                L[i] = L[i - 1];
            } else {
                L[i] = x;
                placed = true;
            }
        }
    }
    if (!placed)
        L[0] = x;
}

// k rounds of block arg-max over list heads; results to out (k entries).
__device__ void block_extract(VK (&L)[TK_LIST], int k, VK *out)
{
    __shared__ VK s_best[TK_THREADS / 32];
    __shared__ int s_who[TK_THREADS / 32];
    __shared__ int s_win;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < k; r++) {
        VK b = L[0];
        int who = threadIdx.x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            VK ob;
            ob.v = __shfl_xor_sync(0xffffffffu, b.v, o);
            ob.k = __shfl_xor_sync(0xffffffffu, b.k, o);
            int ow = __shfl_xor_sync(0xffffffffu, who, o);
            if (better(ob, b) || (!better(b, ob) && ow < who)) {
                b = ob;
                who = ow;
            }
        }
        if (lane == 0) {
            s_best[warp] = b;
            s_who[warp] = who;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            VK bb = s_best[0];
            int ww = s_who[0];
            for (int w = 1; w < TK_THREADS / 32; w++)
                if (better(s_best[w], bb) || (!better(bb, s_best[w]) && s_who[w] < ww)) {
                    bb = s_best[w];
                    ww = s_who[w];
                }
            out[r] = bb;
            s_win = ww;
        }
        __syncthreads();
        if (threadIdx.x == s_win) {
#pragma unroll
            for (int i = 0; i < TK_LIST - 1; i++)
                L[i] = L[i + 1];
            L[TK_LIST - 1] = worst_vk();
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TK_THREADS) topk_pass1_kernel(const long long *__restrict__ vals,
                                                                const int32_t *__restrict__ keys, long long n_max,
                                                                const long long *d_n, int k, VK *cand)
{
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    VK L[TK_LIST];
#pragma unroll
    for (int i = 0; i < TK_LIST; i++)
        L[i] = worst_vk();
    for (long long i = (long long)blockIdx.x * TK_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * TK_THREADS) {
        VK x;
        x.v = vals[i];
        x.k = keys[i];
        list_insert(L, x);
    }
    block_extract(L, k, cand + (size_t)blockIdx.x * k);
}

__global__ void __launch_bounds__(TK_THREADS) topk_pass2_kernel(const VK *__restrict__ cand, long long ncand,
                                                                long long n_max, const long long *d_n, int k,
                                                                long long *out_vals, int32_t *out_keys, long long *d_k)
{
    __shared__ VK s_out[TK_MAXK];
    VK L[TK_LIST];
#pragma unroll
    for (int i = 0; i < TK_LIST; i++)
        L[i] = worst_vk();
    for (long long i = threadIdx.x; i < ncand; i += TK_THREADS)
        list_insert(L, cand[i]);
    block_extract(L, k, s_out);
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
    long long want = (n + TK_THREADS * 16 - 1) / (TK_THREADS * 16);
    return (int)std::max(1ll, std::min<long long>(want, (long long)num_sms() * 2));
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_topk_workspace(int64_t n, int32_t k)
{
    if (k < 1 || k > TK_MAXK)
        return 0;
    return align_up((size_t)topk_blocks(n) * k * sizeof(VK), 256);
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
    VK *cand = (VK *)ws;
    topk_pass1_kernel<<<blocks, TK_THREADS, 0, s>>>((const long long *)vals, keys, n, (const long long *)d_n, k, cand);
    topk_pass2_kernel<<<1, TK_THREADS, 0, s>>>(cand, (long long)blocks * k, n, (const long long *)d_n, k,
                                               (long long *)out_vals, out_keys, (long long *)d_k);
    return launch_status();
}
