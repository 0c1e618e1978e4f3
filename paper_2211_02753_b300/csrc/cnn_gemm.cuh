// BF16 tensor-core GEMM core of the glyph-CNN kernels.
//
// C[m][n] = sum_k A(m, k) * B(n, k), FP32 accumulation, mma.sync m16n8k16
// (bf16 inputs) fed by ldmatrix.  Each operand is staged in shared memory in
// the layout its global source has: K-major ([row][k], k contiguous; plain
// ldmatrix) or MN-major ([k][row], row contiguous; ldmatrix.trans builds the
// same fragments), so no operand is ever transposed in global memory.  Tiles
// move in 16-byte chunks, either with cp.async (a plain address per chunk, or
// zero fill) or through registers when the chunk is computed (a virtual
// operand, e.g. the gradient of a max-pool expanded from the pooled gradient
// and its arg-max).  Three pipeline stages.  The epilogue is a functor that
// receives the accumulators of each thread with their (m, n) coordinates.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace tdp {
namespace cnn {

constexpr int GBK = 32;     // k per stage
constexpr int GSTAGES = 3;  // pipeline depth
constexpr int GTHREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    uint32_t s = smem_u32(smem);
    int sz = valid ? 16 : 0; // src-size 0: zero fill
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

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory tile geometry of one operand with `ROWS` rows (m or n).
template <int ROWS, bool MN_MAJOR>
struct TileGeom {
    // K-major: [ROWS][GBK + 8] (row pitch 80 B); MN-major: [GBK][ROWS + 8].
    static constexpr int PITCH = MN_MAJOR ? ROWS + 8 : GBK + 8;
    static constexpr int ELEMS = MN_MAJOR ? GBK * PITCH : ROWS * PITCH;
    static constexpr int CHUNKS = ROWS * GBK / 8; // 16-byte chunks per stage
    // chunk c -> (r, kc) for K-major (kc = k/8) or (k, rc) for MN-major (rc = row/8)
    __device__ static __forceinline__ void chunk_coord(int c, int &a, int &b)
    {
        if (MN_MAJOR) {
            a = c / (ROWS / 8); // k
            b = c % (ROWS / 8); // row chunk
        } else {
            a = c / (GBK / 8);  // row
            b = c % (GBK / 8);  // k chunk
        }
    }
    __device__ static __forceinline__ int chunk_offset(int a, int b)
    {
        return MN_MAJOR ? a * PITCH + b * 8 : a * PITCH + b * 8;
    }
};

// Operand loader concept:
//   static constexpr bool MN_MAJOR;
//   static constexpr bool REG;            // chunk computed in registers
//   cp.async form:  __device__ const void *ptr(int row, int k8, int m0_or_n0, int k0) (nullptr: zero)
//      -- for MN-major: ptr(k, row8, ...) with row8 the 8-row chunk index
//   register form:  __device__ uint4 val(int a, int b, int row0, int k0)
template <int BM, int BN, int WM, int WN, class LA, class LB, class EPI>
__global__ void __launch_bounds__(GTHREADS) gemm_kernel(LA la, LB lb, EPI epi, int M, int N, int K, int k_per_split)
{
    static_assert(WM * WN == GTHREADS / 32, "warp grid");
    constexpr int TM = BM / WM;       // warp tile m
    constexpr int TN = BN / WN;       // warp tile n
    constexpr int FM = TM / 16;       // m16 fragments per warp
    constexpr int FN = TN / 8;        // n8 fragments per warp
    static_assert(FM >= 1 && FN >= 2 && FN % 2 == 0, "warp tile");
    using GA = TileGeom<BM, LA::MN_MAJOR>;
    using GB = TileGeom<BN, LB::MN_MAJOR>;
    extern __shared__ __align__(16) __nv_bfloat16 gsm[];
    __nv_bfloat16 *sA = gsm;
    __nv_bfloat16 *sB = gsm + GSTAGES * GA::ELEMS;

    const int m0 = blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * k_per_split;
    const int kend = min(K, kbeg + k_per_split);
    const int ktiles = (kend - kbeg + GBK - 1) / GBK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp / WN, wn = warp % WN;

    auto load_stage = [&](int stage, int kt) {
        const int k0 = kbeg + kt * GBK;
        __nv_bfloat16 *a = sA + stage * GA::ELEMS;
        __nv_bfloat16 *b = sB + stage * GB::ELEMS;
        for (int c = tid; c < GA::CHUNKS; c += GTHREADS) {
            int x, y;
            GA::chunk_coord(c, x, y);
            void *dst = a + GA::chunk_offset(x, y);
            if constexpr (LA::REG) {
                *(uint4 *)dst = la.val(x, y, m0, k0, kend);
            } else {
                const void *src = la.ptr(x, y, m0, k0, kend);
                cp_async16(dst, src, src != nullptr);
            }
        }
        for (int c = tid; c < GB::CHUNKS; c += GTHREADS) {
            int x, y;
            GB::chunk_coord(c, x, y);
            void *dst = b + GB::chunk_offset(x, y);
            if constexpr (LB::REG) {
                *(uint4 *)dst = lb.val(x, y, n0, k0, kend);
            } else {
                const void *src = lb.ptr(x, y, n0, k0, kend);
                cp_async16(dst, src, src != nullptr);
            }
        }
    };

    float acc[FM][FN][4];
#pragma unroll
    for (int i = 0; i < FM; i++)
#pragma unroll
        for (int j = 0; j < FN; j++)
#pragma unroll
            for (int r = 0; r < 4; r++)
                acc[i][j][r] = 0.f;

#pragma unroll
    for (int s = 0; s < GSTAGES - 1; s++) {
        if (s < ktiles)
            load_stage(s, s);
        cp_async_commit();
    }
    const int li = lane >> 3, lr = lane & 7;
    for (int kt = 0; kt < ktiles; kt++) {
        cp_async_wait<GSTAGES - 2>();
        __syncthreads();
        {
            int nk = kt + GSTAGES - 1;
            if (nk < ktiles)
                load_stage(nk % GSTAGES, nk);
            cp_async_commit();
        }
        const __nv_bfloat16 *a = sA + (kt % GSTAGES) * GA::ELEMS;
        const __nv_bfloat16 *b = sB + (kt % GSTAGES) * GB::ELEMS;
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[FM][4];
#pragma unroll
            for (int i = 0; i < FM; i++) {
                const int mr = wm * TM + i * 16;
                if constexpr (LA::MN_MAJOR) {
                    // matrices (m+0,k+0) (m+8,k+0) (m+0,k+8) (m+8,k+8), stored [k][m]
                    int k = kk + lr + (li >> 1) * 8, m = mr + (li & 1) * 8;
                    ldsm_x4_t(smem_u32(a + k * GA::PITCH + m), af[i][0], af[i][1], af[i][2], af[i][3]);
                } else {
                    int m = mr + (lane & 15), k = kk + (lane >> 4) * 8;
                    ldsm_x4(smem_u32(a + m * GA::PITCH + k), af[i][0], af[i][1], af[i][2], af[i][3]);
                }
            }
#pragma unroll
            for (int j = 0; j < FN; j += 2) {
                const int nr = wn * TN + j * 8;
                uint32_t b0, b1, b2, b3;
                if constexpr (LB::MN_MAJOR) {
                    // (n+0,k+0) (n+0,k+8) (n+8,k+0) (n+8,k+8), stored [k][n]
                    int k = kk + lr + (li & 1) * 8, n = nr + (li >> 1) * 8;
                    ldsm_x4_t(smem_u32(b + k * GB::PITCH + n), b0, b1, b2, b3);
                } else {
                    int n = nr + lr + (li >> 1) * 8, k = kk + (li & 1) * 8;
                    ldsm_x4(smem_u32(b + n * GB::PITCH + k), b0, b1, b2, b3);
                }
#pragma unroll
                for (int i = 0; i < FM; i++) {
                    mma_bf16(acc[i][j], af[i], b0, b1);
                    mma_bf16(acc[i][j + 1], af[i], b2, b3);
                }
            }
        }
    }
    cp_async_wait<0>();
    // epilogue: thread holds rows (g, g+8) x cols (2t, 2t+1) of each fragment
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < FM; i++)
#pragma unroll
        for (int j = 0; j < FN; j++) {
            const int m = m0 + wm * TM + i * 16 + g;
            const int n = n0 + wn * TN + j * 8 + 2 * t;
            epi(m, n, acc[i][j][0], acc[i][j][1], blockIdx.z);
            epi(m + 8, n, acc[i][j][2], acc[i][j][3], blockIdx.z);
        }
    (void)M;
    (void)N;
}

template <int BM, int BN, bool AMN, bool BMN>
constexpr size_t gemm_smem()
{
    return (size_t)GSTAGES * (TileGeom<BM, AMN>::ELEMS + TileGeom<BN, BMN>::ELEMS) * 2;
}

} // namespace cnn
} // namespace tdp
