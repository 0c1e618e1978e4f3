// Soft ORDER BY ... LIMIT k: logistic soft ranks within groups, soft top-k
// membership and sums, their backward, and the exact ranks (Sec. 4's
// relaxation of comparisons applied to a rank).
//
// Every rank is a sum over the row's group, so the work is pairwise: a block
// takes 256 rows of one group (grid: groups x row tiles), stages the
// group's scores through shared memory in chunks, and each thread adds the
// logistic comparisons of its row with every row of the chunk.  A logistic
// costs two special-function operations (2^x and 1/x), the pipe that bounds
// these kernels; the scores are staged pre-scaled by log2(e) / tau so a
// comparison is one subtraction away from 2^x.  fp32 partials of 32 terms are
// added with Kahan compensation (B300's float64 pipe is far too slow to take
// one add per 32 terms at this rate), so a rank over a thousand rows keeps
// about 1e-4 of absolute accuracy.
#include <algorithm>

#include "common.cuh"
#include "tdp_softsort.h"

namespace tdp {
namespace softsort {

constexpr int SS_THREADS = 256;
constexpr int SS_CH = 2048; // scores per staged chunk

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated (Kahan) accumulation of fp32 partial sums.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// sigma(u) without overflow either way
__device__ __forceinline__ float sigmoid(float u)
{
    const float e = expf(-fabsf(u));
    const float a = 1.0f / (1.0f + e);
    return u >= 0.f ? a : e * a;
}

// The group's row range; false (and TDP_ERR_CAPACITY) for a malformed or
// oversized group.
__device__ __forceinline__ bool group_rows(const int64_t *__restrict__ offsets, long long g, long long n,
                                           long long max_group, long long &a, long long &b, int32_t *d_status)
{
    a = offsets[g];
    b = offsets[g + 1];
    if (a < 0 || b < a || b > n || b - a > max_group) {
        if (threadIdx.x == 0 && blockIdx.y == 0)
            set_status(d_status, TDP_ERR_CAPACITY);
        return false;
    }
    return true;
}

// MODE 0: soft ranks and membership.  MODE 1: exact ranks.
template <int MODE>
__global__ void __launch_bounds__(SS_THREADS) ss_rank_kernel(const float *__restrict__ x, long long n,
                                                             const int64_t *__restrict__ offsets, long long max_group,
                                                             float c, float kh, float inv_tau_r,
                                                             float *__restrict__ rank_f, float *__restrict__ mask,
                                                             int32_t *__restrict__ rank_i, int32_t *d_status)
{
    __shared__ __align__(16) float sx[SS_CH];
    long long a, b;
    if (!group_rows(offsets, blockIdx.x, n, max_group, a, b, d_status))
        return;
    const int ng = (int)(b - a);
    const int base = blockIdx.y * SS_THREADS;
    if (base >= ng)
        return; // the whole tile lies past the group (uniform exit)
    const int il = base + threadIdx.x;
    const bool valid = il < ng;
    const float xi = valid ? x[a + il] : 0.f;
    const float xc = xi * c;
    Kahan acc;
    int cnt = 0;
    for (int c0 = 0; c0 < ng; c0 += SS_CH) {
        const int m = min(SS_CH, ng - c0);
        for (int t = threadIdx.x; t < m; t += SS_THREADS)
            sx[t] = MODE == 0 ? x[a + c0 + t] * c : x[a + c0 + t];
        __syncthreads();
        if (valid) {
            if (MODE == 0) {
                int j = 0;
                for (; j + 32 <= m; j += 32) {
                    float p = 0.f;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        const float4 s4 = *reinterpret_cast<const float4 *>(sx + j + q);
                        p += rcp_approx(1.0f + ex2_approx(xc - s4.x));
                        p += rcp_approx(1.0f + ex2_approx(xc - s4.y));
                        p += rcp_approx(1.0f + ex2_approx(xc - s4.z));
                        p += rcp_approx(1.0f + ex2_approx(xc - s4.w));
                    }
                    acc.add(p);
                }
                float p = 0.f;
                for (; j < m; j++)
                    p += rcp_approx(1.0f + ex2_approx(xc - sx[j]));
                acc.add(p);
            } else {
                for (int j = 0; j < m; j++) {
                    const float xj = sx[j];
                    cnt += (xj > xi) || (xj == xi && c0 + j < il);
                }
            }
        }
        __syncthreads();
    }
    if (!valid)
        return;
    if (MODE == 0) {
        // the sum ran over j == i too: take out that term, computed the same way
        const float sii = rcp_approx(1.0f + ex2_approx(xc - xc));
        acc.add(-sii);
        const float r = 1.0f + (acc.s - acc.c);
        rank_f[a + il] = r;
        mask[a + il] = sigmoid((kh - r) * inv_tau_r);
    } else {
        rank_i[a + il] = 1 + cnt;
    }
}

// Per group: sum of mask * v (soft) or of v over rank <= k (exact), each
// thread's rows in order in float64, then a fixed tree over the threads.
template <int MODE>
__global__ void __launch_bounds__(SS_THREADS) ss_group_sum_kernel(const float *__restrict__ v,
                                                                  const float *__restrict__ mask,
                                                                  const int32_t *__restrict__ rank_i, int k,
                                                                  long long n, const int64_t *__restrict__ offsets,
                                                                  long long max_group, float *__restrict__ sum_f,
                                                                  double *__restrict__ sum_d, int32_t *d_status)
{
    __shared__ double sred[SS_THREADS];
    long long a, b;
    const long long g = blockIdx.x;
    if (!group_rows(offsets, g, n, max_group, a, b, d_status)) {
        if (threadIdx.x == 0) {
            if (MODE == 0)
                sum_f[g] = 0.f;
            else
                sum_d[g] = 0.0;
        }
        return;
    }
    double s = 0.0;
    for (long long i = a + threadIdx.x; i < b; i += SS_THREADS)
        s += MODE == 0 ? (double)mask[i] * (double)v[i] : (rank_i[i] <= k ? (double)v[i] : 0.0);
    sred[threadIdx.x] = s;
    __syncthreads();
    for (int h = SS_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            sred[threadIdx.x] += sred[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (MODE == 0)
            sum_f[g] = (float)sred[0];
        else
            sum_d[g] = sred[0];
    }
}

// Backward, per row: dm = dsum[g] v + dmask, dr = -dm m (1 - m) / tau_r + drank,
// dv = dsum[g] m.
__global__ void __launch_bounds__(SS_THREADS) ss_bwd_prep_kernel(const float *__restrict__ v,
                                                                 const float *__restrict__ mask, long long n,
                                                                 const int64_t *__restrict__ offsets,
                                                                 long long max_group, float inv_tau_r,
                                                                 const float *__restrict__ dsum,
                                                                 const float *__restrict__ dmask,
                                                                 const float *__restrict__ drank,
                                                                 float *__restrict__ dr, float *__restrict__ dv,
                                                                 int32_t *d_status)
{
    long long a, b;
    const long long g = blockIdx.x;
    if (!group_rows(offsets, g, n, max_group, a, b, d_status))
        return;
    const float ds = dsum ? dsum[g] : 0.f;
    for (long long i = a + threadIdx.x; i < b; i += SS_THREADS) {
        const float m = mask[i];
        const float dm = (dsum && v ? ds * v[i] : 0.f) + (dmask ? dmask[i] : 0.f);
        dr[i] = -dm * m * (1.f - m) * inv_tau_r + (drank ? drank[i] : 0.f);
        if (dv)
            dv[i] = ds * m;
    }
}

// dx_i = (1 / tau) sum_j sigma'(u_ij) (dr_j - dr_i), sigma'(u) = e s^2 with
// e = e^-u = 2^-z and s = 1 / (1 + e).  The j == i terms of the two sums
// cancel, so they are not skipped.  2^-z is capped at 2^64 (there
// sigma' < 2^-64) so that e s^2 never forms inf * 0.
__global__ void __launch_bounds__(SS_THREADS) ss_bwd_pair_kernel(const float *__restrict__ x,
                                                                 const float *__restrict__ dr, long long n,
                                                                 const int64_t *__restrict__ offsets,
                                                                 long long max_group, float c, float inv_tau,
                                                                 float *__restrict__ dx, int32_t *d_status)
{
    __shared__ __align__(16) float sx[SS_CH];
    __shared__ __align__(16) float sd[SS_CH];
    long long a, b;
    if (!group_rows(offsets, blockIdx.x, n, max_group, a, b, d_status))
        return;
    const int ng = (int)(b - a);
    const int base = blockIdx.y * SS_THREADS;
    if (base >= ng)
        return;
    const int il = base + threadIdx.x;
    const bool valid = il < ng;
    const float xc = valid ? x[a + il] * c : 0.f;
    const float di = valid ? dr[a + il] : 0.f;
    Kahan A, Bs;
    for (int c0 = 0; c0 < ng; c0 += SS_CH) {
        const int m = min(SS_CH, ng - c0);
        for (int t = threadIdx.x; t < m; t += SS_THREADS) {
            sx[t] = x[a + c0 + t] * c;
            sd[t] = dr[a + c0 + t];
        }
        __syncthreads();
        if (valid) {
            int j = 0;
            for (; j + 32 <= m; j += 32) {
                float pa = 0.f, pb = 0.f;
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const float4 s4 = *reinterpret_cast<const float4 *>(sx + j + q);
                    const float4 d4 = *reinterpret_cast<const float4 *>(sd + j + q);
                    const float sv[4] = {s4.x, s4.y, s4.z, s4.w}, dv4[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const float e = ex2_approx(fminf(xc - sv[u], 64.f));
                        const float s = rcp_approx(1.0f + e);
                        const float w = e * s * s;
                        pa = fmaf(w, dv4[u], pa);
                        pb += w;
                    }
                }
                A.add(pa);
                Bs.add(pb);
            }
            float pa = 0.f, pb = 0.f;
            for (; j < m; j++) {
                const float e = ex2_approx(fminf(xc - sx[j], 64.f));
                const float s = rcp_approx(1.0f + e);
                const float w = e * s * s;
                pa = fmaf(w, sd[j], pa);
                pb += w;
            }
            A.add(pa);
            Bs.add(pb);
        }
        __syncthreads();
    }
    if (valid)
        dx[a + il] = ((A.s - A.c) - di * (Bs.s - Bs.c)) * inv_tau;
}

} // namespace softsort
} // namespace tdp

using namespace tdp;
using namespace tdp::softsort;

namespace {

constexpr double LOG2E = 1.4426950408889634;

bool ss_args_ok(const float *x, int64_t n, const int64_t *offsets, int64_t n_groups, int64_t max_group, int32_t k)
{
    return n >= 0 && n_groups >= 0 && k >= 1 && max_group >= 1 && max_group <= (1ll << 24) &&
           n_groups <= 0x7fffffffll && (n_groups == 0 || (x && offsets));
}

dim3 ss_grid(int64_t n_groups, int64_t max_group)
{
    return dim3((unsigned)n_groups, (unsigned)((max_group + SS_THREADS - 1) / SS_THREADS));
}

} // namespace

extern "C" {

tdp_status tdp_soft_topk_fwd(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                             int64_t max_group, int32_t k, float tau, float tau_r, float *rank, float *mask,
                             float *sum, int32_t *d_status, tdp_stream_t stream)
{
    if (!ss_args_ok(x, n, offsets, n_groups, max_group, k) || !(tau > 0.f) || !(tau_r > 0.f) ||
        (n_groups > 0 && (!rank || !mask)) || (sum && !v))
        return TDP_ERR_INVALID_ARG;
    if (n_groups == 0)
        return TDP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ss_rank_kernel<0><<<ss_grid(n_groups, max_group), SS_THREADS, 0, s>>>(
        x, n, offsets, max_group, (float)(LOG2E / tau), (float)k + 0.5f, 1.0f / tau_r, rank, mask, nullptr,
        d_status);
    if (sum)
        ss_group_sum_kernel<0><<<(unsigned)n_groups, SS_THREADS, 0, s>>>(v, mask, nullptr, k, n, offsets, max_group,
                                                                         sum, nullptr, d_status);
    return launch_status();
}

size_t tdp_soft_topk_workspace(int64_t n) { return align_up((size_t)std::max<int64_t>(n, 1) * sizeof(float), 256); }

tdp_status tdp_soft_topk_bwd(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                             int64_t max_group, int32_t k, float tau, float tau_r, const float *mask,
                             const float *dsum, const float *dmask, const float *drank, float *dx, float *dv,
                             void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (!ss_args_ok(x, n, offsets, n_groups, max_group, k) || !(tau > 0.f) || !(tau_r > 0.f) ||
        (n_groups > 0 && (!mask || !dx)) || (dsum && !v) || (dv && !dsum))
        return TDP_ERR_INVALID_ARG;
    if (n_groups == 0)
        return TDP_OK;
    if (!ws || (uintptr_t)ws % 16 || ws_bytes < tdp_soft_topk_workspace(n))
        return ws && (uintptr_t)ws % 16 ? TDP_ERR_INVALID_ARG : TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    float *dr = (float *)ws;
    ss_bwd_prep_kernel<<<(unsigned)n_groups, SS_THREADS, 0, s>>>(v, mask, n, offsets, max_group, 1.0f / tau_r, dsum,
                                                                 dmask, drank, dr, dv, d_status);
    ss_bwd_pair_kernel<<<ss_grid(n_groups, max_group), SS_THREADS, 0, s>>>(x, dr, n, offsets, max_group,
                                                                           (float)(LOG2E / tau), 1.0f / tau, dx,
                                                                           d_status);
    return launch_status();
}

tdp_status tdp_exact_topk(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                          int64_t max_group, int32_t k, int32_t *rank, double *sum, int32_t *d_status,
                          tdp_stream_t stream)
{
    if (!ss_args_ok(x, n, offsets, n_groups, max_group, k) || (n_groups > 0 && !rank) || (sum && !v))
        return TDP_ERR_INVALID_ARG;
    if (n_groups == 0)
        return TDP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ss_rank_kernel<1><<<ss_grid(n_groups, max_group), SS_THREADS, 0, s>>>(x, n, offsets, max_group, 1.f, 0.f, 0.f,
                                                                          nullptr, nullptr, rank, d_status);
    if (sum)
        ss_group_sum_kernel<1><<<(unsigned)n_groups, SS_THREADS, 0, s>>>(v, nullptr, rank, k, n, offsets, max_group,
                                                                         nullptr, sum, d_status);
    return launch_status();
}

} // extern "C"
