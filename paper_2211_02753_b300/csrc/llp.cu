// Learning from label proportions (Sec. 5.3) and its label-DP counts
// (Sec. 5.4): the bags' count labels, one fused forward + backward pass of
// the linear classifier's soft bag COUNT, and the hard classifier.
//
// The step kernel reads X once.  Rows are taken in groups of whole bags (as
// many bags as fit in one staged chunk of LLP_CH rows, or one bag when a bag
// is longer than that); a block stages its group's rows in shared memory
// with coalesced loads, computes every row's class probabilities, sums them
// per bag in a fixed order, forms each bag's count gradient from its own
// target right there, and accumulates the weight gradient from the staged
// rows.  Blocks are persistent (a grid of at most the resident count) and
// write one partial row each; a one-block kernel adds the rows in float64 in
// a fixed order.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "tdp_llp.h"

namespace tdp {
namespace llp {

constexpr int LLP_THREADS = 256;
constexpr int LLP_WARPS = LLP_THREADS / 32;
constexpr int LLP_CH = 1024;     // rows per staged chunk
constexpr int LLP_MAX_BLOCKS_PER_SM = 8;

// partial row: dW [K][d], db [K], loss
__host__ __device__ inline int part_len(int K, int d) { return K * d + K + 1; }

__device__ __forceinline__ void stage_rows(const float *__restrict__ src, long long nf, float *__restrict__ dst)
{
    const int tid = threadIdx.x;
    if (((uintptr_t)src & 15) == 0) {
        const long long n4 = nf >> 2;
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (long long i = tid; i < n4; i += LLP_THREADS)
            d4[i] = __ldcs(s4 + i);
        for (long long i = (n4 << 2) + tid; i < nf; i += LLP_THREADS)
            dst[i] = __ldcs(src + i);
    } else {
        for (long long i = tid; i < nf; i += LLP_THREADS)
            dst[i] = __ldcs(src + i);
    }
}

// class probabilities of one staged row
template <int KM, int DM>
__device__ __forceinline__ void row_probs(const float *__restrict__ x, const float *__restrict__ sW,
                                          const float *__restrict__ sb, int K, int d, float (&P)[KM])
{
    float mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < KM; k++) {
        float s = 0.f;
        if (k < K) {
            s = sb[k];
#pragma unroll
            for (int f = 0; f < DM; f++)
                if (f < d)
                    s = fmaf(x[f], sW[k * DM + f], s);
            mx = fmaxf(mx, s);
        }
        P[k] = s;
    }
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < KM; k++) {
        P[k] = k < K ? expf(P[k] - mx) : 0.f;
        z += P[k];
    }
    const float iz = 1.0f / z;
#pragma unroll
    for (int k = 0; k < KM; k++)
        P[k] *= iz;
}

// gradient of one row: dl = P (dP - <P, dP>), dW += dl x^T, db += dl
template <int KM, int DM>
__device__ __forceinline__ void row_grad(const float *__restrict__ x, const float (&P)[KM],
                                         const float *__restrict__ dP, int K, int d, float (&acc)[KM][DM],
                                         float (&accb)[KM])
{
    float dot = 0.f;
#pragma unroll
    for (int k = 0; k < KM; k++)
        if (k < K)
            dot = fmaf(P[k], dP[k], dot);
#pragma unroll
    for (int k = 0; k < KM; k++) {
        if (k < K) {
            const float dl = P[k] * (dP[k] - dot);
            accb[k] += dl;
#pragma unroll
            for (int f = 0; f < DM; f++)
                if (f < d)
                    acc[k][f] = fmaf(dl, x[f], acc[k][f]);
        }
    }
}

// A bag's counts are final: its loss share, its count gradient, the counts out.
template <int KM>
__device__ __forceinline__ void finish_bag(const float (&c)[KM], long long bag, int K,
                                           const float *__restrict__ target, float inv_nout,
                                           float *__restrict__ cnt_out, float *__restrict__ dc, float &accl)
{
#pragma unroll
    for (int k = 0; k < KM; k++) {
        if (k < K) {
            const float dd = c[k] - target[bag * K + k];
            accl = fmaf(dd, dd, accl);
            dc[k] = 2.f * dd * inv_nout;
            if (cnt_out)
                cnt_out[bag * K + k] = c[k];
        }
    }
}

template <int KM, int DM>
__global__ void __launch_bounds__(LLP_THREADS) llp_step_kernel(const float *__restrict__ X, long long n, int d, int K,
                                                               long long B, const float *__restrict__ W,
                                                               const float *__restrict__ bias,
                                                               const float *__restrict__ target, float inv_nout,
                                                               float *__restrict__ cnt_out, float *__restrict__ part,
                                                               long long G, long long ngroups)
{
    extern __shared__ float4 llp_smem[];
    float *sX = reinterpret_cast<float *>(llp_smem); // [LLP_CH][d]
    float *sP = sX + LLP_CH * d;                      // [LLP_CH][KM]
    float *sdc = sP + LLP_CH * KM;                    // [bags of the group][KM]
    __shared__ float sW[KM * DM], sb[KM];
    __shared__ float sred[LLP_WARPS][KM * DM + KM + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < KM * DM; i += LLP_THREADS) {
        const int k = i / DM, f = i % DM;
        sW[i] = (k < K && f < d) ? W[k * d + f] : 0.f;
    }
    if (tid < KM)
        sb[tid] = tid < K ? bias[tid] : 0.f;
    float acc[KM][DM], accb[KM], accl = 0.f;
#pragma unroll
    for (int k = 0; k < KM; k++) {
        accb[k] = 0.f;
#pragma unroll
        for (int f = 0; f < DM; f++)
            acc[k][f] = 0.f;
    }
    __syncthreads();

    for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const long long r0 = g * G;
        const long long rows = min(G, n - r0);
        if (G <= LLP_CH) {
            // ---- whole bags in one chunk
            const int nr = (int)rows, Bi = (int)B;
            stage_rows(X + r0 * d, (long long)nr * d, sX);
            __syncthreads();
            for (int r = tid; r < nr; r += LLP_THREADS) {
                float P[KM];
                row_probs<KM, DM>(sX + r * d, sW, sb, K, d, P);
#pragma unroll
                for (int k = 0; k < KM; k++)
                    sP[r * KM + k] = P[k];
            }
            __syncthreads();
            const int nb = (nr + Bi - 1) / Bi;
            const long long bag0 = r0 / B;
            if (Bi <= 32) { // a thread per bag, rows in order
                for (int j = tid; j < nb; j += LLP_THREADS) {
                    float c[KM];
#pragma unroll
                    for (int k = 0; k < KM; k++)
                        c[k] = 0.f;
                    const int re = min(nr, (j + 1) * Bi);
                    for (int r = j * Bi; r < re; r++)
#pragma unroll
                        for (int k = 0; k < KM; k++)
                            c[k] += sP[r * KM + k];
                    finish_bag<KM>(c, bag0 + j, K, target, inv_nout, cnt_out, sdc + j * KM, accl);
                }
            } else { // a warp per bag: lane-strided sums, then a fixed xor tree
                for (int j = warp; j < nb; j += LLP_WARPS) {
                    float c[KM];
#pragma unroll
                    for (int k = 0; k < KM; k++)
                        c[k] = 0.f;
                    const int re = min(nr, (j + 1) * Bi);
                    for (int r = j * Bi + lane; r < re; r += 32)
#pragma unroll
                        for (int k = 0; k < KM; k++)
                            c[k] += sP[r * KM + k];
#pragma unroll
                    for (int k = 0; k < KM; k++)
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1)
                            c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
                    if (lane == 0)
                        finish_bag<KM>(c, bag0 + j, K, target, inv_nout, cnt_out, sdc + j * KM, accl);
                }
            }
            __syncthreads();
            for (int r = tid; r < nr; r += LLP_THREADS) {
                float P[KM];
#pragma unroll
                for (int k = 0; k < KM; k++)
                    P[k] = sP[r * KM + k];
                row_grad<KM, DM>(sX + r * d, P, sdc + (r / Bi) * KM, K, d, acc, accb);
            }
            __syncthreads(); // the next group restages sX, sP and sdc
        } else {
            // ---- one bag longer than a chunk: sum its probabilities chunk by
            // chunk, then stage the chunks again for the gradient
            float c[KM];
#pragma unroll
            for (int k = 0; k < KM; k++)
                c[k] = 0.f;
            for (long long c0 = 0; c0 < rows; c0 += LLP_CH) {
                const int nr = (int)min((long long)LLP_CH, rows - c0);
                stage_rows(X + (r0 + c0) * d, (long long)nr * d, sX);
                __syncthreads();
                for (int r = tid; r < nr; r += LLP_THREADS) {
                    float P[KM];
                    row_probs<KM, DM>(sX + r * d, sW, sb, K, d, P);
#pragma unroll
                    for (int k = 0; k < KM; k++)
                        c[k] += P[k];
                }
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < KM; k++) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
                if (lane == 0)
                    sP[warp * KM + k] = c[k];
            }
            __syncthreads();
            if (tid == 0) {
                float t[KM];
#pragma unroll
                for (int k = 0; k < KM; k++) {
                    t[k] = 0.f;
                    for (int w = 0; w < LLP_WARPS; w++)
                        t[k] += sP[w * KM + k];
                }
                finish_bag<KM>(t, r0 / B, K, target, inv_nout, cnt_out, sdc, accl);
            }
            __syncthreads();
            float dP[KM];
#pragma unroll
            for (int k = 0; k < KM; k++)
                dP[k] = sdc[k];
            for (long long c0 = 0; c0 < rows; c0 += LLP_CH) {
                const int nr = (int)min((long long)LLP_CH, rows - c0);
                __syncthreads(); // sX of the previous chunk fully used
                stage_rows(X + (r0 + c0) * d, (long long)nr * d, sX);
                __syncthreads();
                for (int r = tid; r < nr; r += LLP_THREADS) {
                    float P[KM];
                    row_probs<KM, DM>(sX + r * d, sW, sb, K, d, P);
                    row_grad<KM, DM>(sX + r * d, P, dP, K, d, acc, accb);
                }
            }
            __syncthreads();
        }
    }

    // ---- block partial: warp xor trees, then the warps in order
    const int per = part_len(K, d);
#pragma unroll
    for (int k = 0; k < KM; k++) {
#pragma unroll
        for (int f = 0; f < DM; f++) {
            float v = acc[k][f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && k < K && f < d)
                sred[warp][k * d + f] = v;
        }
        float v = accb[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && k < K)
            sred[warp][K * d + k] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        accl += __shfl_xor_sync(0xffffffffu, accl, o);
    if (lane == 0)
        sred[warp][K * d + K] = accl * inv_nout;
    __syncthreads();
    for (int v = tid; v < per; v += LLP_THREADS) {
        float s = 0.f;
        for (int w = 0; w < LLP_WARPS; w++)
            s += sred[w][v];
        part[(size_t)blockIdx.x * per + v] = s;
    }
}

// ---------------------------------------------------------------------------
// Streaming step for two classes and at most 8 features (the census shape).
//
// With two classes the softmax depends on the logit gap only,
// P1 = sigma(z1 - z0), and the logit gradient of a row is
// dl0 = P0 (dc0 - P0 dc0 - P1 dc1) = P0 P1 (dc0 - dc1) = -dl1, where dc is
// its bag's count gradient.  So the weight gradient factors per bag:
//   dW[0] = sum_bags delta_b S_b,  db[0] = sum_bags delta_b T_b,
//   S_b = sum_{i in b} P0_i P1_i x_i,  T_b = sum_{i in b} P0_i P1_i,
//   delta_b = dc0_b - dc1_b = 2 (e0_b - e1_b) / (n_bags K),  e = cnt - target,
// and dW[1] = -dW[0], db[1] = -db[0].  Every bag needs only sums over its
// rows (cnt0, cnt1, T, S), so one pass over X suffices and no row is
// visited twice.
//
// Each warp works alone on one contiguous range of rows made of whole tasks
// (tasks of whole bags, split evenly over the warps).  It streams the range
// through its own ring of LLP_NST shared-memory stages of LLP_SR rows,
// filled by bulk copies that lane 0 issues LLP_NST stages ahead, and its
// lanes take one row each per step of 32 rows.  Bags of a multiple of 32
// rows are whole steps; bags of a divisor of 32 rows are aligned lane
// groups.  Only a bag's two counts are reduced across its lanes (they give
// delta); S and T stay per-lane partials scaled by delta, and the lanes'
// gradient sums meet once, at the end.  No block barrier is taken until the
// final partial sums.
constexpr int LLP_ST = 256;         // threads of the streaming kernel
constexpr int LLP_SW = LLP_ST / 32; // its warps
constexpr int LLP_SR = 128;         // rows per stage
constexpr int LLP_NST = 3;          // stages in a warp's ring
constexpr int LLP_TASK = 512;       // rows per task (whole bags; a bag longer than this is one task)

__host__ __device__ inline long long task_rows(long long B)
{
    return B <= LLP_TASK ? (LLP_TASK / B) * B : B;
}

__device__ __forceinline__ void issue_stage(float *buf, const float *X, long long r0, int rows, int d, uint64_t *bar)
{
    const uint32_t bytes16 = (uint32_t)(rows * d * 4) & ~15u;
    mbar_arrive_expect_tx(bar, bytes16);
    if (bytes16)
        bulk_load(buf, X + r0 * d, bytes16, bar);
}

// A bag's counts c0, c1 are final (every lane of the bag holds them): its
// count error against the target, and each lane's share of the gradient,
// delta * (its partial S, T).  The bag's leader adds the loss and writes the
// counts.
template <int DM>
__device__ __forceinline__ void finish_bag2(long long bag, bool leader, float c0, float c1, float T,
                                            const float (&S)[DM], const float *__restrict__ target, float two_inv,
                                            float *__restrict__ cnt_out, float (&gW)[DM], float &gb, float &gl)
{
    const float2 t = __ldg(reinterpret_cast<const float2 *>(target) + bag);
    const float e0 = c0 - t.x, e1 = c1 - t.y;
    const float delta = two_inv * (e0 - e1);
    gb = fmaf(delta, T, gb);
#pragma unroll
    for (int f = 0; f < DM; f++)
        gW[f] = fmaf(delta, S[f], gW[f]);
    if (leader) {
        gl = fmaf(e0, e0, fmaf(e1, e1, gl));
        if (cnt_out)
            reinterpret_cast<float2 *>(cnt_out)[bag] = make_float2(c0, c1);
    }
}

// One step: each lane's row of the 32 (FULL: all rows present) adds to the
// lane's running sums of P0, P1, T = P0 P1 and S = P0 P1 x.
template <int DM, bool FULL>
__device__ __forceinline__ void step_rows(const float *__restrict__ buf, int rr, int rows, int d,
                                          const float (&w)[DM], float bd, float &c0, float &c1, float &T,
                                          float (&S)[DM])
{
    if (!FULL && rr >= rows)
        return;
    float x[DM];
    const float *xr = buf + rr * d;
    if ((d & 1) == 0) {
#pragma unroll
        for (int f = 0; f < DM; f += 2) {
            if (f < d) {
                const float2 v = *reinterpret_cast<const float2 *>(xr + f);
                x[f] = v.x;
                x[f + 1] = v.y;
            } else {
                x[f] = x[f + 1] = 0.f;
            }
        }
    } else {
#pragma unroll
        for (int f = 0; f < DM; f++)
            x[f] = f < d ? xr[f] : 0.f;
    }
    float dz = bd;
#pragma unroll
    for (int f = 0; f < DM; f++)
        dz = fmaf(x[f], w[f], dz);
    // P1 = sigma(z1 - z0) from e = 2^-|dz2| in (0, 1] (no overflow either
    // way); 1 + e lies in [1, 2], where the fast divide holds
    const float e = exp2f(-fabsf(dz));
    const float a = __fdividef(1.0f, 1.0f + e);
    const float P0 = dz >= 0.f ? e * a : a;
    const float P1 = dz >= 0.f ? a : e * a;
    const float h = P0 * P1;
    c0 += P0;
    c1 += P1;
    T += h;
#pragma unroll
    for (int f = 0; f < DM; f++)
        S[f] = fmaf(h, x[f], S[f]);
}

template <int DM, bool EXACT>
__global__ void __launch_bounds__(LLP_ST) llp_stream_kernel(const float *__restrict__ X, long long n, int d_rt,
                                                           long long B, const float *__restrict__ W,
                                                           const float *__restrict__ bias,
                                                           const float *__restrict__ target, float inv_nout,
                                                           float *__restrict__ cnt_out, float *__restrict__ part,
                                                           long long ntasks, int32_t *d_status, uint32_t spin)
{
    extern __shared__ float4 llp_smem[];
    const int d = EXACT ? DM : d_rt; // row width (a constant when the kernel is built for it)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *ring = reinterpret_cast<float *>(llp_smem) + (size_t)warp * LLP_NST * LLP_SR * d;
    __shared__ uint64_t bar[LLP_SW][LLP_NST];
    __shared__ float sred[LLP_SW][DM + 2];
    // the logit gap in base 2: dz2 = log2(e) (z1 - z0), so e^-|dz| = 2^-|dz2|
    constexpr float LOG2E = 1.4426950408889634f;
    float w[DM];
#pragma unroll
    for (int f = 0; f < DM; f++)
        w[f] = f < d ? (W[d + f] - W[f]) * LOG2E : 0.f;
    const float bd = (bias[1] - bias[0]) * LOG2E;
    const float two_inv = 2.f * inv_nout;
    const bool big = B % 32 == 0; // else B divides 32 (a power of two)
    const int lgB = big ? 0 : __ffs((int)B) - 1;
    const int Bi = (int)B;        // bags of the streamed path hold at most 2^30 rows

    // this warp's rows: tasks [gw * ntasks / nw, (gw + 1) * ntasks / nw)
    const long long TR = task_rows(B);
    const long long nw = (long long)gridDim.x * LLP_SW, gw = (long long)blockIdx.x * LLP_SW + warp;
    const long long wbeg = min(n, (gw * ntasks / nw) * TR), wend = min(n, ((gw + 1) * ntasks / nw) * TR);
    const int nstages = (int)((wend - wbeg + LLP_SR - 1) / LLP_SR);

    if (lane == 0)
        for (int q = 0; q < LLP_NST; q++)
            mbar_init(&bar[warp][q], 1);
    __syncwarp();
    if (lane == 0)
        for (int q = 0; q < LLP_NST && q < nstages; q++) {
            const long long r0 = wbeg + (long long)q * LLP_SR;
            issue_stage(ring + q * LLP_SR * d, X, r0, (int)min((long long)LLP_SR, wend - r0), d, &bar[warp][q]);
        }

    float gW[DM], gb = 0.f, gl = 0.f;
    float S[DM], c0 = 0.f, c1 = 0.f, T = 0.f;
#pragma unroll
    for (int f = 0; f < DM; f++)
        gW[f] = S[f] = 0.f;
    long long bag = big ? wbeg / B : 0; // the next bag to finish (bags of a multiple of 32 rows)
    int rib = 0;                        // rows of that bag seen so far
    int it = 0;
    bool failed = false;
    for (; it < nstages; it++) {
        const int q = it % LLP_NST;
        float *buf = ring + q * LLP_SR * d;
        const long long r0 = wbeg + (long long)it * LLP_SR;
        const int rows = (int)min((long long)LLP_SR, wend - r0);
        const bool ok = mbar_wait_sleep(&bar[warp][q], (uint32_t)(it / LLP_NST) & 1u, spin);
        if (!__all_sync(0xffffffffu, ok)) {
            failed = true;
            break;
        }
        const int tail = rows * d - (int)(((uint32_t)(rows * d * 4) & ~15u) >> 2); // < 4 floats not copied
        if (tail) {
            if (lane < tail) {
                buf[rows * d - tail + lane] = X[r0 * d + rows * d - tail + lane];
                fence_proxy_async_smem(); // before the stage is refilled by a bulk copy
            }
            __syncwarp();
        }
        const bool full = rows == LLP_SR;
#pragma unroll
        for (int st = 0; st < LLP_SR; st += 32) {
            if (st >= rows)
                break;
            if (full)
                step_rows<DM, true>(buf, st + lane, rows, d, w, bd, c0, c1, T, S);
            else
                step_rows<DM, false>(buf, st + lane, rows, d, w, bd, c0, c1, T, S);
            bool done; // a bag (or, for bags that divide 32, every lane group) ends with this step
            if (big) {
                rib += 32;
                done = rib == Bi || st + 32 >= rows && it + 1 == nstages; // full, or the last rows
            } else {
                done = true;
                for (int o = Bi >> 1; o > 0; o >>= 1) {
                    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
                }
            }
            if (big && done) {
                // only the counts are reduced across the warp; S and T stay
                // lane partials, scaled by the bag's delta
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
                }
                finish_bag2<DM>(bag, lane == 0, c0, c1, T, S, target, two_inv, cnt_out, gW, gb, gl);
                bag++;
                rib = 0;
            } else if (!big) {
                const int lead = st + (lane & ~(Bi - 1)); // the lane group's first row in this stage
                if (lead < rows)
                    finish_bag2<DM>((r0 + lead) >> lgB, (lane & (Bi - 1)) == 0, c0, c1, T, S, target, two_inv,
                                    cnt_out, gW, gb, gl);
            }
            if (done) {
                c0 = c1 = T = 0.f;
#pragma unroll
                for (int f = 0; f < DM; f++)
                    S[f] = 0.f;
            }
        }
        // the stage has been read: lane 0 refills it LLP_NST stages ahead
        __syncwarp();
        if (lane == 0 && it + LLP_NST < nstages) {
            const long long pr0 = wbeg + (long long)(it + LLP_NST) * LLP_SR;
            fence_proxy_async_smem();
            issue_stage(buf, X, pr0, (int)min((long long)LLP_SR, wend - pr0), d, &bar[warp][q]);
        }
    }
    if (failed) {
        // a wait ran out: report it, and let this warp's copies still in
        // flight land (bounded) before the block's shared memory is released
        if (lane == 0) {
            set_status(d_status, TDP_ERR_TIMEOUT);
            for (int k = it; k < nstages && k < it + LLP_NST; k++)
                mbar_wait_sleep(&bar[warp][k % LLP_NST], (uint32_t)(k / LLP_NST) & 1u, spin);
        }
        gl = gb = 0.f;
#pragma unroll
        for (int f = 0; f < DM; f++)
            gW[f] = 0.f;
    }
    // block partial: warp sums, then the warps in order
#pragma unroll
    for (int f = 0; f < DM; f++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            gW[f] += __shfl_xor_sync(0xffffffffu, gW[f], o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gb += __shfl_xor_sync(0xffffffffu, gb, o);
        gl += __shfl_xor_sync(0xffffffffu, gl, o);
    }
    if (lane == 0) {
#pragma unroll
        for (int f = 0; f < DM; f++)
            sred[warp][f] = gW[f];
        sred[warp][DM] = gb;
        sred[warp][DM + 1] = gl * inv_nout;
    }
    __syncthreads();
    const int per = part_len(2, d);
    float *pp = part + (size_t)blockIdx.x * per;
    if (tid < d + 2) {
        const int v = tid < d ? tid : DM + (tid - d);
        float sum = 0.f;
        for (int k = 0; k < LLP_SW; k++)
            sum += sred[k][v];
        if (tid < d) {
            pp[tid] = sum;
            pp[d + tid] = -sum;
        } else if (tid == d) {
            pp[2 * d] = sum;
            pp[2 * d + 1] = -sum;
        } else {
            pp[2 * d + 2] = sum;
        }
    }
}

// dW, db, loss = the sums of the blocks' partial rows in float64, in a fixed
// order: a warp per column, lane l adds blocks l, l + 32, ... in order, then
// a fixed xor tree over the lanes.
constexpr int LLP_RED_THREADS = 1024;

__global__ void __launch_bounds__(LLP_RED_THREADS) llp_reduce_kernel(const float *__restrict__ part, int nblk, int K,
                                                                     int d, float *__restrict__ dW,
                                                                     float *__restrict__ db, float *__restrict__ loss)
{
    const int per = part_len(K, d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = warp; v < per; v += LLP_RED_THREADS / 32) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32)
            s += part[(size_t)b * per + v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (v < K * d)
                dW[v] = (float)s;
            else if (v < K * d + K)
                db[v - K * d] = (float)s;
            else
                loss[0] = (float)s;
        }
    }
}

// counts[j][k] = #{ labels == k in bag j } + scale * noise[j][k]; one thread
// per (bag, class)
// Bags smaller than a warp: a thread per (bag, class) counts its bag.
__global__ void llp_counts_small_kernel(const int32_t *__restrict__ labels, long long n, int K, long long B,
                                        const float *__restrict__ noise, float scale, float *__restrict__ counts,
                                        int32_t *__restrict__ d_status)
{
    const long long nbags = (n + B - 1) / B;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbags * K)
        return;
    const long long j = i / K;
    const int k = (int)(i % K);
    const long long re = min(n, (j + 1) * B);
    long long c = 0;
    bool bad = false;
    for (long long r = j * B; r < re; r++) {
        const int32_t y = labels[r];
        c += y == k;
        bad |= (k == 0) && (y < 0 || y >= K);
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    counts[i] = noise ? (float)c + scale * noise[i] : (float)c;
}

// Bags of at least a warp's rows: a warp per bag (bags in grid-stride order), its
// lanes reading consecutive labels (coalesced) and counting each class in
// registers; the warp adds the lanes' counts and lane k writes class k.
template <int KM>
__global__ void llp_counts_kernel(const int32_t *__restrict__ labels, long long n, int K, long long B,
                                  const float *__restrict__ noise, float scale, float *__restrict__ counts,
                                  int32_t *__restrict__ d_status)
{
    const long long nbags = (n + B - 1) / B;
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (long long j = w0; j < nbags; j += nw) {
        const long long re = min(n, (j + 1) * B);
        unsigned c[KM];
#pragma unroll
        for (int k = 0; k < KM; k++)
            c[k] = 0;
        for (long long r = j * B + lane; r < re; r += 32) {
            const int32_t y = __ldcs(labels + r);
            bad |= y < 0 || y >= K;
#pragma unroll
            for (int k = 0; k < KM; k++)
                c[k] += y == k;
        }
        unsigned mine = 0;
#pragma unroll
        for (int k = 0; k < KM; k++) {
            const unsigned v = __reduce_add_sync(0xffffffffu, c[k]);
            if (lane == k)
                mine = v;
        }
        if (lane < K) {
            const long long i = j * K + lane;
            counts[i] = noise ? (float)mine + scale * noise[i] : (float)mine;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        set_status(d_status, TDP_ERR_OVERFLOW);
}

template <int KM, int DM>
__global__ void llp_predict_kernel(const float *__restrict__ X, long long n, int d, int K,
                                   const float *__restrict__ W, const float *__restrict__ bias,
                                   int32_t *__restrict__ labels_out, const int32_t *__restrict__ ref,
                                   unsigned long long *__restrict__ d_errors)
{
    __shared__ float sW[KM * DM], sb[KM];
    for (int i = threadIdx.x; i < KM * DM; i += blockDim.x) {
        const int k = i / DM, f = i % DM;
        sW[i] = (k < K && f < d) ? W[k * d + f] : 0.f;
    }
    if (threadIdx.x < KM)
        sb[threadIdx.x] = threadIdx.x < K ? bias[threadIdx.x] : 0.f;
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int wrong = 0;
    if (i < n) {
        float x[DM];
#pragma unroll
        for (int f = 0; f < DM; f++)
            x[f] = f < d ? X[i * d + f] : 0.f;
        int best = 0;
        float bv = 0.f;
#pragma unroll
        for (int k = 0; k < KM; k++) {
            if (k < K) {
                float s = sb[k];
#pragma unroll
                for (int f = 0; f < DM; f++)
                    if (f < d)
                        s = fmaf(x[f], sW[k * DM + f], s);
                if (k == 0 || s > bv) {
                    bv = s;
                    best = k;
                }
            }
        }
        if (labels_out)
            labels_out[i] = best;
        if (ref)
            wrong = ref[i] != best;
    }
    if (ref) {
        const unsigned m = __ballot_sync(0xffffffffu, wrong);
        if ((threadIdx.x & 31) == 0 && m)
            atomicAdd(d_errors, (unsigned long long)__popc(m));
    }
}

} // namespace llp
} // namespace tdp

using namespace tdp;
using namespace tdp::llp;

namespace {

// rows per group: as many whole bags as fit in one chunk, else one bag
long long group_rows(long long B) { return B <= LLP_CH ? (LLP_CH / B) * B : B; }

size_t step_smem(int d, int KM) { return (size_t)LLP_CH * d * 4 + 2 * (size_t)LLP_CH * KM * 4; }

// Resident blocks per SM of the step kernel for d features (queried once per
// d).  The kernel's dynamic shared memory limit is set to what the widest
// row (DM features) needs, never lower, so every d launches under it.
template <int KM, int DM> int step_blocks_per_sm(int d)
{
    static std::atomic<int> cache[DM + 1];
    int v = cache[d].load(std::memory_order_relaxed);
    if (v > 0)
        return v;
    if (cudaFuncSetAttribute(llp_step_kernel<KM, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem(DM, KM)) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, llp_step_kernel<KM, DM>, LLP_THREADS,
                                                      step_smem(d, KM)) != cudaSuccess)
        return -1;
    v = std::max(1, std::min(per_sm, LLP_MAX_BLOCKS_PER_SM));
    cache[d].store(v, std::memory_order_relaxed);
    return v;
}

template <int KM, int DM> int step_grid(long long ngroups, int d)
{
    const int per_sm = step_blocks_per_sm<KM, DM>(d);
    if (per_sm < 1)
        return -1;
    return (int)std::min<long long>(ngroups, (long long)per_sm * num_sms());
}

template <int KM, int DM>
tdp_status launch_step(const float *X, long long n, int d, int K, long long B, const float *W, const float *b,
                       const float *targets, float *cnt, float *loss, float *dW, float *db, float *part,
                       cudaStream_t s)
{
    const long long G = group_rows(B);
    const long long ngroups = (n + G - 1) / G;
    const int grid = step_grid<KM, DM>(ngroups, d);
    if (grid < 1)
        return TDP_ERR_CUDA;
    const long long nbags = (n + B - 1) / B;
    llp_step_kernel<KM, DM><<<grid, LLP_THREADS, step_smem(d, KM), s>>>(
        X, n, d, K, B, W, b, targets, 1.0f / (float)((double)nbags * K), cnt, part, G, ngroups);
    llp_reduce_kernel<<<1, LLP_RED_THREADS, 0, s>>>(part, grid, K, d, dW, db, loss);
    return launch_status();
}

bool dims_ok(int K, int d) { return K >= 2 && K <= 4 && d >= 1 && d <= 16; }

size_t stream_smem(int d) { return (size_t)LLP_SW * LLP_NST * LLP_SR * d * 4; }

// Resident blocks per SM of one streaming kernel (queried once per width;
// the dynamic shared memory limit is set for the widest row).
template <int DM, bool EXACT> int stream_blocks_per_sm(int d)
{
    static std::atomic<int> cache[DM + 1];
    int v = cache[d].load(std::memory_order_relaxed);
    if (v > 0)
        return v;
    if (cudaFuncSetAttribute(llp_stream_kernel<DM, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stream_smem(DM)) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, llp_stream_kernel<DM, EXACT>, LLP_ST,
                                                      stream_smem(d)) != cudaSuccess)
        return -1;
    v = std::max(1, std::min(per_sm, LLP_MAX_BLOCKS_PER_SM));
    cache[d].store(v, std::memory_order_relaxed);
    return v;
}

// The streaming kernel takes two classes, at most 8 features, bags of a
// multiple or a divisor of 32 rows, rows starting on 16-byte boundaries
// (bulk copies of whole stages) and 8-byte aligned targets and counts.
bool stream_ok(const float *X, const float *targets, const float *cnt, int d, int K, long long B)
{
    return K == 2 && d <= 8 && (B % 32 == 0 || 32 % B == 0) && B <= (1ll << 30) && (uintptr_t)X % 16 == 0 &&
           (uintptr_t)targets % 8 == 0 && (uintptr_t)cnt % 8 == 0; // (targets, counts) read and written as pairs
}

tdp_status launch_stream(const float *X, long long n, int d, long long B, const float *W, const float *b,
                         const float *targets, float *cnt, float *loss, float *dW, float *db, float *part,
                         int32_t *d_status, cudaStream_t s)
{
    const long long TR = task_rows(B);
    const long long ntasks = (n + TR - 1) / TR;
    const bool census = d == 6;
    const int per_sm = census ? stream_blocks_per_sm<6, true>(d) : stream_blocks_per_sm<8, false>(d);
    if (per_sm < 1)
        return TDP_ERR_CUDA;
    const long long want = (ntasks + LLP_SW - 1) / LLP_SW;
    const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)per_sm * num_sms()));
    const long long nbags = (n + B - 1) / B;
    const float inv = 1.0f / (float)((double)nbags * 2);
    if (census)
        llp_stream_kernel<6, true><<<grid, LLP_ST, stream_smem(d), s>>>(X, n, d, B, W, b, targets, inv, cnt, part,
                                                                       ntasks, d_status, spin_limit());
    else
        llp_stream_kernel<8, false><<<grid, LLP_ST, stream_smem(d), s>>>(X, n, d, B, W, b, targets, inv, cnt,
                                                                        part, ntasks, d_status, spin_limit());
    llp_reduce_kernel<<<1, LLP_RED_THREADS, 0, s>>>(part, grid, 2, d, dW, db, loss);
    return launch_status();
}

} // namespace

extern "C" {

tdp_status tdp_llp_counts(const int32_t *labels, int64_t n, int32_t K, int64_t B, const float *noise, float scale,
                          float *counts, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || K < 1 || K > 16 || B < 1 || (n > 0 && (!labels || !counts)))
        return TDP_ERR_INVALID_ARG;
    if (n == 0)
        return TDP_OK;
    const long long nbags = (n + B - 1) / B;
    if (B < 32) {
        const long long work = nbags * K;
        llp_counts_small_kernel<<<(unsigned)((work + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            labels, n, K, B, noise, scale, counts, d_status);
        return launch_status();
    }
    const unsigned grid = (unsigned)std::max(1ll, std::min<long long>((nbags + 7) / 8, (long long)num_sms() * 16));
    if (K <= 2)
        llp_counts_kernel<2><<<grid, 256, 0, (cudaStream_t)stream>>>(labels, n, K, B, noise, scale, counts, d_status);
    else
        llp_counts_kernel<16><<<grid, 256, 0, (cudaStream_t)stream>>>(labels, n, K, B, noise, scale, counts,
                                                                       d_status);
    return launch_status();
}

size_t tdp_llp_step_workspace(int64_t n, int32_t d, int32_t K, int64_t B)
{
    if (n < 1 || B < 1 || !dims_ok(K, d))
        return 0;
    const long long G = group_rows(B);
    const long long ngroups = (n + G - 1) / G;
    const long long blocks = std::min<long long>(ngroups, (long long)LLP_MAX_BLOCKS_PER_SM * num_sms());
    return align_up((size_t)blocks * part_len(K, d) * sizeof(float), 256);
}

tdp_status tdp_llp_step(const float *X, int64_t n, int32_t d, int32_t K, int64_t B, const float *W, const float *b,
                        const float *targets, float *cnt, float *loss, float *dW, float *db, void *ws,
                        size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || B < 1 || !dims_ok(K, d))
        return TDP_ERR_INVALID_ARG;
    if (n > 0 && (!X || !W || !b || !targets || !loss || !dW || !db))
        return TDP_ERR_INVALID_ARG;
    if ((uintptr_t)X % 4)
        return TDP_ERR_INVALID_ARG;
    if (n == 0)
        return TDP_OK;
    if (ws && (uintptr_t)ws % 16)
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_llp_step_workspace(n, d, K, B))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    float *part = (float *)ws;
    if (stream_ok(X, targets, cnt, d, K, B))
        return launch_stream(X, n, d, B, W, b, targets, cnt, loss, dW, db, part, d_status, s);
    if (K <= 2 && d <= 8)
        return launch_step<2, 8>(X, n, d, K, B, W, b, targets, cnt, loss, dW, db, part, s);
    return launch_step<4, 16>(X, n, d, K, B, W, b, targets, cnt, loss, dW, db, part, s);
}

tdp_status tdp_llp_predict(const float *X, int64_t n, int32_t d, int32_t K, const float *W, const float *b,
                           int32_t *labels_out, const int32_t *ref_labels, int64_t *d_errors, tdp_stream_t stream)
{
    if (n < 0 || !dims_ok(K, d) || (n > 0 && (!X || !W || !b)) || (ref_labels && !d_errors))
        return TDP_ERR_INVALID_ARG;
    if (n == 0)
        return TDP_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    if (K <= 2 && d <= 8)
        llp_predict_kernel<2, 8><<<blocks, 256, 0, s>>>(X, n, d, K, W, b, labels_out, ref_labels,
                                                        (unsigned long long *)d_errors);
    else
        llp_predict_kernel<4, 16><<<blocks, 256, 0, s>>>(X, n, d, K, W, b, labels_out, ref_labels,
                                                         (unsigned long long *)d_errors);
    return launch_status();
}

} // extern "C"
