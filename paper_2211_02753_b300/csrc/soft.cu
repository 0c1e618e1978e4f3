// K9/K10: soft filter and soft grouped aggregation with hand-written adjoints
// (Sec. 4: logistic relaxation of a predicate, soft_count / soft_groupby).
//
// Rows stream through once per call with 16-byte loads (x, v: float4; gid:
// int4).  Each block owns a contiguous chunk of rows and accumulates per-group
// sums in shared memory as compensated fp32 pairs (hi, lo): each row's term t
// goes to hi by an fp32 atomic add, whose returned old value gives the exact
// rounding error of old + t by TwoSum (Knuth), and that error goes to lo by a
// second atomic.  hi + lo then carries the block's sum to about fp32^2
// relative accuracy whatever the order of the atomics.  The per-block sums
// are then added in fp64, in block order, by a second small kernel.
// (Upstream gradients of either sign make the adjoint's group sums cancel;
// plain fp32 sub-sums, even of ~16 rows per group, left the cancelling groups
// of the adjoint at the edge of the 1e-5 bound, and fp64 shared-memory
// atomics cost twice the time of the whole kernel.)
// The mask m = sigmoid((x - theta[g]) / tau) is recomputed in the backward
// pass, never stored; m(1-m) is evaluated as e/(1+e)^2 with e = exp(-|z|),
// which has no cancellation when m is close to 1.  z = (x - theta) / tau is
// carried as a pair zh + zl (x - theta by TwoSum, the division's residual by
// an FMA) and exp(-|z|) is corrected to first order in zl: the exponential
// multiplies the rounding error of a plain fp32 z by |z| (up to ~50 at
// tau = 0.1), which alone used most of the 1e-5 budget of the adjoint.
#include <atomic>

#include "common.cuh"

namespace tdp {

constexpr int SA_THREADS = 512;
constexpr int SA_UNROLL = 2;        // row quads a thread loads ahead
constexpr int SA_BLOCKS_PER_SM = 3; // resident blocks the register budget allows
constexpr int SA_MAX_GROUPS = 4096;

struct Sig {
    float m;  // sigmoid(z)
    float dm; // m (1 - m)
};

struct Tau {
    float t;   // tau
    float inv; // 1 / tau, rounded
};

// sigmoid((x - th) / tau) and its m (1 - m), z = zh + zl as described above.
__device__ __forceinline__ Sig sigmoid_xt(float x, float th, Tau tau)
{
    const float d = x - th;
    const float bb = d - x;
    const float dl = (x - (d - bb)) + (-th - bb); // x - th = d + dl exactly
    const float zh = d * tau.inv;
    const float zl = (fmaf(-zh, tau.t, d) + dl) * tau.inv; // (d + dl - zh tau) / tau
    const float e = expf(-fabsf(zh)) * (1.0f - (zh >= 0.f ? zl : -zl));
    const float r = 1.0f / (1.0f + e);
    Sig s;
    s.m = zh >= 0.f ? r : e * r;
    s.dm = e * r * r;
    return s;
}

enum SoftMode { MODE_AGG_FWD = 0, MODE_AGG_BWD = 1, MODE_FILTER_BWD = 2 };

// acc[0][g] + acc[1][g] += t, compensated (see the header).  An fp32 atomic
// add rounds to nearest, so the value it stores is the fp32 sum old + t, and
// TwoSum recovers that sum's error exactly (no multiply, so nothing fuses).
__device__ __forceinline__ void comp_add(float *hi, int G, int g, float t)
{
    const float old = atomicAdd(&hi[g], t);
    const float sum = old + t;
    const float bt = sum - old;
    const float err = (old - (sum - bt)) + (t - bt);
    atomicAdd(&hi[G + g], err);
}

// Per-row work of the three reduction modes.  Accumulates into the
// compensated shared-memory pairs acc0 (and acc1 for the forward COUNT), each
// laid out [hi: G][lo: G].
template <int MODE>
__device__ __forceinline__ void soft_row(float x, float v, int g, float gm, const float *s_theta, const float *s_g0,
                                         const float *s_g1, Tau tau, float *acc0, float *acc1, float *gx,
                                         float *gv, long long i, int G)
{
    if ((unsigned)g >= (unsigned)G) // out-of-range group id: row ignored
        return;
    Sig s = sigmoid_xt(x, s_theta[g], tau);
    if (MODE == MODE_AGG_FWD) {
        comp_add(acc0, G, g, v * s.m);
        comp_add(acc1, G, g, s.m);
    } else if (MODE == MODE_AGG_BWD) {
        float gS = s_g0[g];
        float w = (gS * v + s_g1[g]) * s.dm;
        comp_add(acc0, G, g, w);
        if (gx)
            gx[i] = w * tau.inv;
        if (gv)
            gv[i] = gS * s.m;
    } else {
        float w = gm * s.dm;
        comp_add(acc0, G, g, w);
        if (gx)
            gx[i] = w * tau.inv;
    }
}

template <int MODE>
__global__ void __launch_bounds__(SA_THREADS, SA_BLOCKS_PER_SM) soft_reduce_kernel(const float *__restrict__ x,
                                                                 const float *__restrict__ v,
                                                                 const int32_t *__restrict__ gid,
                                                                 const float *__restrict__ theta,
                                                                 const float *__restrict__ g0,
                                                                 const float *__restrict__ g1, Tau tau,
                                                                 long long n, int G, long long chunk,
                                                                 double *__restrict__ partial, float *gx, float *gv)
{
    // Shared memory: K compensated accumulators [K][hi, lo][G], then theta
    // (and, for the aggregation adjoint, the upstream gradients).
    constexpr int K = MODE == MODE_AGG_FWD ? 2 : 1;
    extern __shared__ float smf[];
    float *acc0 = smf;                       // [2][G]
    float *acc1 = smf + 2 * G;               // [2][G], forward COUNT only
    float *s_theta = smf + 2 * K * G;
    float *s_g0 = s_theta + G;               // aggregation backward only
    float *s_g1 = s_theta + 2 * G;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        s_theta[g] = theta[g];
        acc0[g] = acc0[G + g] = 0.f;
        if (MODE == MODE_AGG_FWD)
            acc1[g] = acc1[G + g] = 0.f;
        if (MODE == MODE_AGG_BWD) {
            s_g0[g] = g0[g];
            s_g1[g] = g1[g];
        }
    }
    __syncthreads();
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    const bool vec = (((uintptr_t)x | (uintptr_t)gid | (uintptr_t)(MODE == MODE_FILTER_BWD ? g0 : v)) % 16) == 0;
    const float *aux = MODE == MODE_FILTER_BWD ? g0 : v; // v, or grad_mask for the filter adjoint
    long long tail = beg;
    if (vec && beg < end) {
        const long long nvec = (end - beg) / 4;
        // SA_UNROLL quads a thread per pass, all of their loads issued
        // before any row is reduced (bytes in flight for the HBM)
        long long q = threadIdx.x;
        for (; q + (SA_UNROLL - 1) * SA_THREADS < nvec; q += SA_UNROLL * SA_THREADS) {
            float4 xx[SA_UNROLL], aa[SA_UNROLL];
            int4 gg[SA_UNROLL];
#pragma unroll
            for (int u = 0; u < SA_UNROLL; u++) {
                const long long i = beg + 4 * (q + u * SA_THREADS);
                xx[u] = __ldcs((const float4 *)(x + i));
                aa[u] = __ldcs((const float4 *)(aux + i));
                gg[u] = __ldcs((const int4 *)(gid + i));
            }
#pragma unroll
            for (int u = 0; u < SA_UNROLL; u++) {
                const long long i = beg + 4 * (q + u * SA_THREADS);
                soft_row<MODE>(xx[u].x, aa[u].x, gg[u].x, aa[u].x, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i, G);
                soft_row<MODE>(xx[u].y, aa[u].y, gg[u].y, aa[u].y, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 1, G);
                soft_row<MODE>(xx[u].z, aa[u].z, gg[u].z, aa[u].z, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 2, G);
                soft_row<MODE>(xx[u].w, aa[u].w, gg[u].w, aa[u].w, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 3, G);
            }
        }
        for (; q < nvec; q += SA_THREADS) {
            const long long i = beg + 4 * q;
            float4 xx = __ldcs((const float4 *)(x + i));
            float4 aa = __ldcs((const float4 *)(aux + i));
            int4 gg = __ldcs((const int4 *)(gid + i));
            soft_row<MODE>(xx.x, aa.x, gg.x, aa.x, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i, G);
            soft_row<MODE>(xx.y, aa.y, gg.y, aa.y, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 1, G);
            soft_row<MODE>(xx.z, aa.z, gg.z, aa.z, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 2, G);
            soft_row<MODE>(xx.w, aa.w, gg.w, aa.w, s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, i + 3, G);
        }
        tail = beg + 4 * nvec;
    }
    for (long long r = tail + threadIdx.x; r < end; r += SA_THREADS)
        soft_row<MODE>(x[r], aux[r], gid[r], aux[r], s_theta, s_g0, s_g1, tau, acc0, acc1, gx, gv, r, G);
    __syncthreads();
    double *out = partial + (size_t)blockIdx.x * K * G;
    for (int e = threadIdx.x; e < K * G; e += blockDim.x) {
        const int k = e / G, g = e - k * G;
        out[e] = (double)smf[2 * k * G + g] + (double)smf[(2 * k + 1) * G + g];
    }
}

// out[k][g] = scale * sum_b partial[b][k][g] in float64, in a fixed order:
// slice s (of SC_SLICES) sums blocks b = s, s + SC_SLICES, ... in order, then
// the slices are added by a fixed tree.  A block covers 32 consecutive
// (k, g) entries (coalesced loads), each with SC_SLICES threads.
constexpr int SC_SLICES = 16;

__global__ void __launch_bounds__(32 * SC_SLICES) soft_combine_kernel(const double *__restrict__ partial, int nblocks,
                                                                      int G, int K, float scale,
                                                                      float *__restrict__ out0,
                                                                      float *__restrict__ out1)
{
    __shared__ double s_acc[SC_SLICES][32];
    const int e = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + e;
    double acc = 0.0;
    if (t < K * G) {
        int b = sl;
        for (; b + 3 * SC_SLICES < nblocks; b += 4 * SC_SLICES) {
            const double a0 = partial[(size_t)b * K * G + t];
            const double a1 = partial[(size_t)(b + SC_SLICES) * K * G + t];
            const double a2 = partial[(size_t)(b + 2 * SC_SLICES) * K * G + t];
            const double a3 = partial[(size_t)(b + 3 * SC_SLICES) * K * G + t];
            acc += a0;
            acc += a1;
            acc += a2;
            acc += a3;
        }
        for (; b < nblocks; b += SC_SLICES)
            acc += partial[(size_t)b * K * G + t];
    }
    s_acc[sl][e] = acc;
    __syncthreads();
#pragma unroll
    for (int h = SC_SLICES / 2; h > 0; h >>= 1) {
        if (sl < h)
            s_acc[sl][e] += s_acc[sl + h][e];
        __syncthreads();
    }
    if (sl == 0 && t < K * G) {
        const double r = s_acc[0][e] * (double)scale;
        if (t < G)
            out0[t] = (float)r;
        else
            out1[t - G] = (float)r;
    }
}

static inline unsigned combine_blocks(int K, int G) { return (unsigned)((K * G + 31) / 32); }

__global__ void soft_filter_fwd_kernel(const float *__restrict__ x, const int32_t *__restrict__ gid,
                                       const float *__restrict__ theta, Tau tau, long long n,
                                       float *__restrict__ mask)
{
    long long i = 4ll * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    const bool vec = (((uintptr_t)x | (uintptr_t)gid | (uintptr_t)mask) % 16) == 0;
    if (vec && i + 3 < n) {
        float4 xx = __ldg((const float4 *)(x + i));
        int4 gg = __ldg((const int4 *)(gid + i));
        float4 o;
        o.x = sigmoid_xt(xx.x, __ldg(theta + gg.x), tau).m;
        o.y = sigmoid_xt(xx.y, __ldg(theta + gg.y), tau).m;
        o.z = sigmoid_xt(xx.z, __ldg(theta + gg.z), tau).m;
        o.w = sigmoid_xt(xx.w, __ldg(theta + gg.w), tau).m;
        *(float4 *)(mask + i) = o;
    } else {
        for (long long r = i; r < min(n, i + 4); r++)
            mask[r] = sigmoid_xt(x[r], theta[gid[r]], tau).m;
    }
}

struct SoftGrid {
    int blocks;
    long long chunk;
    size_t smem;
};

// n32 fp32 arrays of G entries in shared memory
static SoftGrid soft_grid(long long n, int G, int n32)
{
    SoftGrid sg;
    sg.smem = (size_t)G * n32 * sizeof(float);
    // resident blocks per SM: registers allow SA_BLOCKS_PER_SM, shared memory as it allows
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(SA_BLOCKS_PER_SM, (200 * 1024) / std::max<size_t>(sg.smem, 1)));
    long long want = (n + 4ll * SA_THREADS * 8 - 1) / (4ll * SA_THREADS * 8);
    long long maxb = (long long)num_sms() * per_sm;
    sg.blocks = (int)std::max(1ll, std::min(want, maxb));
    sg.chunk = (n + sg.blocks - 1) / sg.blocks;
    sg.chunk = (sg.chunk + 3) / 4 * 4;
    return sg;
}

static tdp_status set_smem(const void *fn, size_t smem)
{
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    return TDP_OK;
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_soft_workspace(int64_t n, int32_t n_groups)
{
    (void)n;
    // per-block fp64 partials: at most SA_BLOCKS_PER_SM blocks per SM, 2
    // arrays of n_groups
    return align_up((size_t)SA_BLOCKS_PER_SM * num_sms() * 2 * (size_t)std::max(1, n_groups) * sizeof(double), 256);
}

static tdp_status soft_check(const float *x, const int32_t *gid, const float *theta, float tau, int64_t n, int32_t G)
{
    if (n < 0 || G <= 0 || G > SA_MAX_GROUPS || !(tau > 0.f) || !theta)
        return TDP_ERR_INVALID_ARG;
    if (n > 0 && (!x || !gid))
        return TDP_ERR_INVALID_ARG;
    return TDP_OK;
}

extern "C" tdp_status tdp_soft_filter_fwd(const float *x, const int32_t *gid, const float *theta, float tau,
                                          int64_t n, float *mask, tdp_stream_t stream)
{
    if (n < 0 || !(tau > 0.f) || (n > 0 && (!x || !gid || !theta || !mask)))
        return TDP_ERR_INVALID_ARG;
    if (n == 0)
        return TDP_OK;
    long long threads = (n + 3) / 4;
    soft_filter_fwd_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        x, gid, theta, Tau{tau, 1.0f / tau}, n, mask);
    return launch_status();
}

extern "C" tdp_status tdp_soft_agg_fwd(const float *x, const float *v, const int32_t *gid, const float *theta,
                                       float tau, int64_t n, int32_t G, float *sum, float *cnt, void *ws,
                                       size_t ws_bytes, tdp_stream_t stream)
{
    tdp_status st = soft_check(x, gid, theta, tau, n, G);
    if (st != TDP_OK)
        return st;
    if (!sum || !cnt || (n > 0 && !v))
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_soft_workspace(n, G))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    SoftGrid sg = soft_grid(n, G, 5);
    if ((st = set_smem((const void *)soft_reduce_kernel<MODE_AGG_FWD>, sg.smem)) != TDP_OK)
        return st;
    double *partial = (double *)ws;
    soft_reduce_kernel<MODE_AGG_FWD><<<sg.blocks, SA_THREADS, sg.smem, s>>>(
        x, v, gid, theta, nullptr, nullptr, Tau{tau, 1.0f / tau}, n, G, sg.chunk, partial, nullptr, nullptr);
    soft_combine_kernel<<<combine_blocks(2, G), 32 * SC_SLICES, 0, s>>>(partial, sg.blocks, G, 2, 1.0f, sum, cnt);
    return launch_status();
}

extern "C" tdp_status tdp_soft_agg_bwd(const float *x, const float *v, const int32_t *gid, const float *theta,
                                       float tau, int64_t n, int32_t G, const float *gsum, const float *gcnt,
                                       float *grad_theta, float *grad_v, float *grad_x, void *ws, size_t ws_bytes,
                                       tdp_stream_t stream)
{
    tdp_status st = soft_check(x, gid, theta, tau, n, G);
    if (st != TDP_OK)
        return st;
    if (!gsum || !gcnt || !grad_theta || (n > 0 && !v))
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_soft_workspace(n, G))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    SoftGrid sg = soft_grid(n, G, 5);
    if ((st = set_smem((const void *)soft_reduce_kernel<MODE_AGG_BWD>, sg.smem)) != TDP_OK)
        return st;
    double *partial = (double *)ws;
    soft_reduce_kernel<MODE_AGG_BWD><<<sg.blocks, SA_THREADS, sg.smem, s>>>(
        x, v, gid, theta, gsum, gcnt, Tau{tau, 1.0f / tau}, n, G, sg.chunk, partial, grad_x, grad_v);
    soft_combine_kernel<<<combine_blocks(1, G), 32 * SC_SLICES, 0, s>>>(partial, sg.blocks, G, 1, -1.0f / tau,
                                                                           grad_theta, nullptr);
    return launch_status();
}

extern "C" tdp_status tdp_soft_filter_bwd(const float *x, const int32_t *gid, const float *theta, float tau,
                                          int64_t n, int32_t G, const float *grad_mask, float *grad_x,
                                          float *grad_theta, void *ws, size_t ws_bytes, tdp_stream_t stream)
{
    tdp_status st = soft_check(x, gid, theta, tau, n, G);
    if (st != TDP_OK)
        return st;
    if (!grad_theta || (n > 0 && !grad_mask))
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_soft_workspace(n, G))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    SoftGrid sg = soft_grid(n, G, 3);
    if ((st = set_smem((const void *)soft_reduce_kernel<MODE_FILTER_BWD>, sg.smem)) != TDP_OK)
        return st;
    double *partial = (double *)ws;
    soft_reduce_kernel<MODE_FILTER_BWD><<<sg.blocks, SA_THREADS, sg.smem, s>>>(
        x, nullptr, gid, theta, grad_mask, nullptr, Tau{tau, 1.0f / tau}, n, G, sg.chunk, partial, grad_x, nullptr);
    soft_combine_kernel<<<combine_blocks(1, G), 32 * SC_SLICES, 0, s>>>(partial, sg.blocks, G, 1, -1.0f / tau,
                                                                           grad_theta, nullptr);
    return launch_status();
}

// ---------------------------------------------------------------------------
// tdp_soft_agg_fwd_noalloc: the soft aggregation forward for callers that
// cannot allocate device memory (for example code running where a
// cudaMalloc would synchronise the device or is not permitted, or a host
// that only hands out pre-registered buffers).  Its scratch -- the fp64
// per-block partial sums -- lives in one fixed array in this library's device
// image instead of a caller workspace.
// ---------------------------------------------------------------------------

namespace tdp {

constexpr int NOALLOC_MAX_GROUPS = 1024;
constexpr int NOALLOC_MAX_BLOCKS = 256;
// the forward's shared memory (5 floats per group) stays under the default
// 48 KiB dynamic limit at the largest group count
static_assert(NOALLOC_MAX_GROUPS * 5 * sizeof(float) <= 48 * 1024, "no-alloc shared memory");

// 256 blocks x 2 sums x 1024 groups x 8 bytes = 4 MiB, resident on every GPU
// that loads this library until the process exits.
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_BLOCKS * 2 * NOALLOC_MAX_GROUPS];

// Device address of g_noalloc_partial, looked up once per device (in host
// code the symbol is only a stand-in, never a device address).
static std::atomic<double *> g_noalloc_ptr[64];

static tdp_status noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return TDP_ERR_CUDA;
    double *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_noalloc_partial) != cudaSuccess || !addr)
            return TDP_ERR_CUDA;
        p = (double *)addr;
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return TDP_OK;
}

} // namespace tdp

extern "C" tdp_status tdp_soft_agg_fwd_noalloc(const float *x, const float *v, const int32_t *gid,
                                               const float *theta, float tau, int64_t n, int32_t G, float *sum,
                                               float *cnt, tdp_stream_t stream)
{
    tdp_status st = soft_check(x, gid, theta, tau, n, G);
    if (st != TDP_OK)
        return st;
    if (!sum || !cnt || (n > 0 && !v))
        return TDP_ERR_INVALID_ARG;
    if (G > NOALLOC_MAX_GROUPS) // beyond the fixed scratch: the caller must use tdp_soft_agg_fwd
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    double *partial = nullptr;
    if ((st = noalloc_scratch(&partial)) != TDP_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    SoftGrid sg = soft_grid(n, G, 5);
    if (sg.blocks > NOALLOC_MAX_BLOCKS) {
        sg.blocks = NOALLOC_MAX_BLOCKS;
        sg.chunk = (n + sg.blocks - 1) / sg.blocks;
        sg.chunk = (sg.chunk + 3) / 4 * 4;
    }
    if ((st = set_smem((const void *)soft_reduce_kernel<MODE_AGG_FWD>, sg.smem)) != TDP_OK)
        return st;
    // every block used overwrites its own K x G partials before the combine
    // reads them, so nothing in the shared scratch has to start at zero
    soft_reduce_kernel<MODE_AGG_FWD><<<sg.blocks, SA_THREADS, sg.smem, s>>>(
        x, v, gid, theta, nullptr, nullptr, Tau{tau, 1.0f / tau}, n, G, sg.chunk, partial, nullptr, nullptr);
    soft_combine_kernel<<<combine_blocks(2, G), 32 * SC_SLICES, 0, s>>>(partial, sg.blocks, G, 2, 1.0f, sum, cnt);
    return launch_status();
}
