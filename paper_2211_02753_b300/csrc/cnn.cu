// K12-K18: the glyph-CNN of the trainable query (Sec. 3 training loop,
// Sec. 4 soft operators on probability-encoded columns, Sec. 5.5).
//
// Layers (cells of 28x28 uint8, read in place from the 112x112 grid images):
//   conv1 3x3 1->32 + ReLU       direct, CUDA cores (K = 9), bf16 NHWC out
//   conv2 3x3 32->64 + ReLU      nine accumulating tcgen05 GEMMs over shifted
//     + 2x2 max-pool             views of one input patch; bias, ReLU, pool
//                                and per-channel arg-max byte in the epilogue
//   fc1 9216->128 + ReLU         tcgen05 GEMM, split-K, bf16 out
//   fc2 128->10, softmax, soft COUNT per class and soft row SUM per grid row,
//   MSE loss and its backward    one block per grid (16 cells), fp32
// Backward: fc1 data gradient (masked by the pooled ReLU) and weight gradient
// (split-K) as tcgen05 GEMMs; conv2 data and weight gradients on tcgen05,
// their A operand the pre-pool gradient expanded from the pooled gradient
// through the arg-max; conv1 weight and bias gradients on CUDA cores; a fused
// Adam step that also refreshes the bf16 copies of the tensor-core weights.
// No operand is transposed in global memory or materialised in im2col form.
#include <cuda.h>

#include "cnn_async.cuh"
#include "common.cuh"
#include "umma.cuh"
#include "tdp_cnn.h"

namespace tdp {
namespace cnn {

using bf16 = __nv_bfloat16;

constexpr int CELL = 28, C1 = 26, C2 = 24, PO = 12;
constexpr int CH1 = 32, CH2 = 64, FEAT = PO * PO * CH2, HID = 128, NCLS = 10;
constexpr int GRID_W = 4, GRID_H = 4, CELLS_PER_GRID = 16;

__device__ __forceinline__ float bf2f(bf16 x) { return __bfloat162float(x); }

// ------------------------------------------------------------------ conv1

// conv1 + ReLU, y1[c][oy][ox][co] = relu(b[co] + sum_k x[oy+ky][ox+kx] w[co][k])
// (fp32, taps in order, rounded once to bf16).  Thread = a horizontal pixel
// pair of one cell (26 is even, so pairs never straddle rows): one broadcast
// 16-byte read of the [tap][co] weights feeds 8 FMAs.  A block's 256 pairs
// are 32 KB of y1, contiguous: staged in shared memory (16-byte chunks
// XOR-swizzled by the pair index, conflict-free both ways) and written with
// full-line stores.
constexpr int C1F_THREADS = 256; // pixel pairs per block
constexpr int PAIRS_PER_CELL = C1 * C1 / 2;

__global__ void __launch_bounds__(C1F_THREADS) conv1_fwd_kernel(const uint8_t *__restrict__ grids, long long npairs,
                                                                const float *__restrict__ w,
                                                                const float *__restrict__ b, bf16 *__restrict__ y1)
{
    __shared__ __align__(16) float sw[9][CH1];
    __shared__ float sb[CH1];
    __shared__ uint4 sout[C1F_THREADS * 8];
    const int tid = threadIdx.x;
    for (int i = tid; i < CH1 * 9; i += C1F_THREADS)
        sw[i % 9][i / 9] = w[i]; // w is [co][ky][kx]
    if (tid < CH1)
        sb[tid] = b[tid];
    __syncthreads();
    const long long q0 = (long long)blockIdx.x * C1F_THREADS, q = q0 + tid;
    if (q < npairs) {
        const long long c = q / PAIRS_PER_CELL;
        const int rem = (int)(q % PAIRS_PER_CELL), oy = rem / (C1 / 2), ox = (rem % (C1 / 2)) * 2;
        const long long g = c / CELLS_PER_GRID;
        const int r = (int)(c % CELLS_PER_GRID) / GRID_W, cc = (int)(c % GRID_W);
        const uint8_t *img = grids + g * (GRID_H * CELL) * (GRID_W * CELL) +
                             (long long)(r * CELL + oy) * (GRID_W * CELL) + cc * CELL + ox;
        float x[3][4];
#pragma unroll
        for (int ky = 0; ky < 3; ky++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                x[ky][j] = (float)img[ky * (GRID_W * CELL) + j] * (1.0f / 255.0f);
#pragma unroll
        for (int cg = 0; cg < CH1 / 8; cg++) {
            float a[2][8];
#pragma unroll
            for (int i = 0; i < 8; i++)
                a[0][i] = a[1][i] = sb[cg * 8 + i];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const float4 wa = *(const float4 *)&sw[k][cg * 8], wb = *(const float4 *)&sw[k][cg * 8 + 4];
                const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const float xv = x[k / 3][k % 3 + p];
#pragma unroll
                    for (int i = 0; i < 8; i++)
                        a[p][i] = fmaf(xv, wv[i], a[p][i]);
                }
            }
#pragma unroll
            for (int p = 0; p < 2; p++) {
                uint4 o;
                __nv_bfloat162 *h = (__nv_bfloat162 *)&o;
#pragma unroll
                for (int i = 0; i < 4; i++)
                    h[i] = __floats2bfloat162_rn(fmaxf(a[p][2 * i], 0.f), fmaxf(a[p][2 * i + 1], 0.f));
                sout[tid * 8 + ((p * 4 + cg) ^ (tid & 7))] = o;
            }
        }
    }
    __syncthreads();
    const long long nchunks = (min(npairs, q0 + C1F_THREADS) - q0) * 8;
    uint4 *dst = (uint4 *)y1 + q0 * 8;
    for (int i = tid; i < nchunks; i += C1F_THREADS) {
        const int t = i >> 3;
        dst[i] = sout[t * 8 + ((i & 7) ^ (t & 7))];
    }
}

// -------------------------------------------------------------- epilogues
//
// Called with 32 consecutive accumulator columns of one output row.  An
// epilogue with PREFETCH also stages a tile of its own input in shared
// memory (cp.async, issued before the main loop) and reads it back there.

struct EpiPartialF32 { // out[split][m][ldo]
    static constexpr bool PREFETCH = false;
    float *out;
    int M, ldo;
    size_t split_stride;
    static constexpr int smem_bytes(int) { return 0; }
    __device__ void prefetch(unsigned char *, int, int, int, int) const {}
    __device__ void finish(const unsigned char *, int, int, int, int) const {}
    __device__ void store(int m, int n, const float (&v)[32], int split, unsigned char *, int, int) const
    {
        if (m >= M)
            return;
        float4 *d = (float4 *)(out + split * split_stride + (size_t)m * ldo + n);
#pragma unroll
        for (int e = 0; e < 8; e++)
            d[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
    }
};

// bf16 out[m][ldo] = v * (mask[m][ldo] > 0); the mask tile (128 rows x BN)
// is staged with a row pitch of BN*2 + 16 bytes (a warp's 16-byte reads of
// 32 rows then hit distinct banks).
struct EpiMaskedBf16 {
    static constexpr bool PREFETCH = true;
    bf16 *out;
    const bf16 *mask;
    int M, ldo;
    static constexpr int pitch(int bn) { return bn * 2 + 16; }
    static constexpr int smem_bytes(int bn) { return 128 * pitch(bn); }
    __device__ void prefetch(unsigned char *buf, int m0, int n0, int bn, int tid) const
    {
        const int cpr = bn / 8; // 16-byte chunks per row
        for (int c = tid; c < 128 * cpr; c += 128) {
            const int r = c / cpr, j = c % cpr, m = m0 + r;
            cnn::cp_async16(buf + r * pitch(bn) + j * 16, m < M ? mask + (size_t)m * ldo + n0 + j * 8 : nullptr,
                            m < M);
        }
    }
    // the masked values replace the mask in shared memory (this thread's row)
    __device__ void store(int m, int n, const float (&v)[32], int, unsigned char *buf, int m0, int n0) const
    {
        if (m >= M)
            return;
        uint4 *mk = (uint4 *)(buf + (m - m0) * pitch_bn + (n - n0) * 2);
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const uint4 mm = mk[h];
            const bf16 *mb = (const bf16 *)&mm;
            __align__(16) bf16 ov[8];
#pragma unroll
            for (int e = 0; e < 8; e++)
                ov[e] = __float2bfloat16_rn(bf2f(mb[e]) > 0.f ? v[8 * h + e] : 0.f);
            mk[h] = *(const uint4 *)ov;
        }
    }
    // then the tile leaves with row-contiguous 16-byte stores (a warp writes
    // whole lines), after every thread's store()
    __device__ void finish(const unsigned char *buf, int m0, int n0, int bn, int tid) const
    {
        const int cpr = bn / 8;
        for (int c = tid; c < 128 * cpr; c += 128) {
            const int r = c / cpr, j = c % cpr;
            if (m0 + r < M)
                *(uint4 *)(out + (size_t)(m0 + r) * ldo + n0 + j * 8) = *(const uint4 *)(buf + r * pitch_bn + j * 16);
        }
    }
    int pitch_bn; // the staging row pitch, pitch(BN) of the launch
};

// ------------------------------------------------ dense GEMM on tcgen05
//
// C[m][n] = sum_k A(m, k) B(n, k) for the fully connected layer: one 128 x BN
// output tile per CTA (and one K range of it under split-K), its fp32
// accumulator in tensor memory (BN columns, TMEM lane = row).  Operands move
// by TMA (cp.async.bulk.tensor, completion counted on an mbarrier) in 64-k
// stages, STAGES deep, straight into the layout the MMA reads:
//   K-major operand ([rows][k] in memory): one copy of R rows x 128 bytes
//     (the whole 64-k stage of each row) with the 128-byte swizzle, read
//     through a SWIZZLE_128B descriptor (SBO 1024 per 8-row atom, +32 bytes
//     per K16 step);
//   MN-major operand ([k][rows]): one copy per 64 rows of 64 k x 128 bytes
//     with the 128-byte swizzle (8 KB: eight 1024-byte atoms along K), read
//     through a swizzled MN-major descriptor (1024 bytes per 8 k, 8192 per
//     64 rows, +2048 bytes per K16 step).
// Rows past the tensor (the M tail) arrive as zeros.  One elected lane of
// warp 0 issues the copies of a stage once the MMAs that last read its slot
// have committed (empty[]); one elected lane of warp 1 issues the four K16
// MMAs of a stage once its copies have landed (full[]); then all four warps
// run the epilogue.  Every wait is bounded (TDP_ERR_TIMEOUT).
constexpr int UG_BM = 128, UG_BK = 64, UG_THREADS = 128;

struct GemmOp {         // one operand as the host describes it
    const void *p;
    long long rows;     // extent along M (or N)
    long long kext;     // extent along K
    long long ld;       // elements between consecutive outer rows in memory
    bool mn_major;      // [k][rows] in memory (else [rows][k])
};

template <bool MN> __host__ __device__ constexpr int ug_op_bytes(int rows) { return rows * UG_BK * 2; }
template <bool MN> __device__ __forceinline__ uint64_t ug_desc(uint32_t a)
{
    return MN ? umma::smem_desc_sw128_mn(a, 1024, 8192) : umma::smem_desc_sw128(a);
}
template <bool MN> __device__ __forceinline__ uint32_t ug_kstep() // 16-byte units per K16
{
    return MN ? 128u : 2u;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];" ::"r"(smem_addr(dst)),
                 "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_addr(bar))
                 : "memory");
}

// The copies of one stage of one operand (rows r0.., k k0..k0+63).
template <bool MN>
__device__ __forceinline__ void ug_tma_stage(const CUtensorMap *map, unsigned char *dst, int rows, int r0, int k0,
                                             uint64_t *bar)
{
    if (MN) {
        for (int a = 0; a < rows / 64; a++) // 64 rows x 64 k, 128-byte swizzle
            tma_load_2d(dst + a * 8192, map, r0 + 64 * a, k0, bar);
    } else {
        tma_load_2d(dst, map, k0, r0, bar); // rows x 64 k, 128-byte swizzle
    }
}

template <int BN, int STAGES, bool AMN, bool BMN, class EPI>
__global__ void __launch_bounds__(UG_THREADS) umma_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                               const __grid_constant__ CUtensorMap tb, EPI epi,
                                                               int K, int k_per_split, int32_t *d_status,
                                                               uint32_t limit)
{
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256 && STAGES >= 2, "tile");
    static_assert(!BMN || BN % 64 == 0, "MN-major operands come in 64-row boxes");
    extern __shared__ __align__(1024) unsigned char ug_smem[];
    __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    constexpr int A_BYTES = ug_op_bytes<AMN>(UG_BM), SB = A_BYTES + ug_op_bytes<BMN>(BN);
    unsigned char *epi_buf = ug_smem + STAGES * SB;
    constexpr uint32_t idesc =
        umma::idesc_bf16_f32(UG_BM, BN) | (AMN ? 1u << 15 : 0u) | (BMN ? 1u << 16 : 0u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UG_BM, n0 = blockIdx.y * BN, split = blockIdx.z;
    const int kbeg = split * k_per_split, kend = min(K, kbeg + k_per_split);
    const int ktiles = kend > kbeg ? (kend - kbeg + UG_BK - 1) / UG_BK : 0;

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], 1);
        }
        mbar_init(&s_done, 1);
        s_err = 0;
    }
    if (warp == 0) {
        umma::tmem_alloc(&s_tmem, BN);
        umma::fence_before_sync();
    }
    if constexpr (EPI::PREFETCH)
        epi.prefetch(epi_buf, m0, n0, BN, tid);
    cnn::cp_async_commit();
    __syncthreads(); // the mbarriers and the tensor-memory address
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem;

    if (warp == 0) { // copies
        if (umma::elect_one()) {
            for (int kt = 0; kt < ktiles; kt++) {
                const int s = kt % STAGES;
                if (kt >= STAGES && !mbar_wait(&s_empty[s], (uint32_t)((kt / STAGES) - 1) & 1u, limit)) {
                    s_err = 1;
                    break;
                }
                unsigned char *st = ug_smem + s * SB;
                const int k0 = kbeg + kt * UG_BK;
                mbar_arrive_expect_tx(&s_full[s], (uint32_t)SB);
                ug_tma_stage<AMN>(&ta, st, UG_BM, m0, k0, &s_full[s]);
                ug_tma_stage<BMN>(&tb, st + A_BYTES, BN, n0, k0, &s_full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) { // MMAs
        if (umma::elect_one()) {
            for (int kt = 0; kt < ktiles; kt++) {
                const int s = kt % STAGES;
                if (!mbar_wait(&s_full[s], (uint32_t)(kt / STAGES) & 1u, limit)) {
                    s_err = 1;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t a = smem_addr(ug_smem + s * SB);
                const uint64_t da = ug_desc<AMN>(a), db = ug_desc<BMN>(a + A_BYTES);
#pragma unroll
                for (int j = 0; j < UG_BK / 16; j++)
                    umma::mma_bf16(tmem, da + ug_kstep<AMN>() * j, db + ug_kstep<BMN>() * j, idesc, kt > 0 || j > 0);
                umma::commit(&s_empty[s]);
            }
            umma::commit(&s_done); // fires once every MMA above has completed
        }
        __syncwarp();
    }
    const bool done = mbar_wait(&s_done, 0, limit);
    if (!done)
        s_err = 1;
    if constexpr (EPI::PREFETCH) {
        cnn::cp_async_wait<0>();
        __syncthreads(); // the staged epilogue input
    }
    umma::fence_after_sync();
    const int m = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
        float v[32];
        if (ktiles > 0) {
            float lo[16], hi[16];
            umma::ld_16cols(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, lo);
            umma::ld_16cols(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cb + 16), hi);
#pragma unroll
            for (int e = 0; e < 16; e++) {
                v[e] = lo[e];
                v[16 + e] = hi[e];
            }
        } else {
#pragma unroll
            for (int e = 0; e < 32; e++)
                v[e] = 0.f; // an empty K range contributes zeros
        }
        epi.store(m, n0 + cb, v, split, epi_buf, m0, n0);
    }
    umma::fence_before_sync();
    __syncthreads();
    if constexpr (EPI::PREFETCH)
        epi.finish(epi_buf, m0, n0, BN, tid);
    if (tid == 0 && s_err)
        set_status(d_status, TDP_ERR_TIMEOUT);
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, BN);
    }
}

// cuTensorMapEncodeTiled, looked up through the runtime once (the library
// takes no link-time dependency on the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// Tensor map of one operand: 2-D, bf16, inner dimension the contiguous one,
// zero fill, 128-byte swizzle; K-major: a box of 64 k x box_outer rows;
// MN-major: a box of 64 rows x box_outer (64) k.
static bool ug_tensor_map(const GemmOp &op, int box_outer, CUtensorMap *map)
{
    const cuuint64_t inner = (cuuint64_t)(op.mn_major ? op.rows : op.kext);
    const cuuint64_t outer = (cuuint64_t)(op.mn_major ? op.kext : op.rows);
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {(cuuint64_t)op.ld * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const EncodeTiledFn encode = encode_tiled();
    if (!encode || (uintptr_t)op.p % 16 || (op.ld * 2) % 16 || inner > (cuuint64_t)op.ld)
        return false;
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(op.p), dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// M x N output (N a multiple of BN), K split into `splits` ranges of whole stages.
template <int BN, int STAGES, bool AMN, bool BMN, class EPI>
static tdp_status launch_umma_gemm(const GemmOp &a, const GemmOp &b, const EPI &epi, int M, int N, int K, int splits,
                                   int32_t *d_status, cudaStream_t s)
{
    if (N % BN || a.mn_major != AMN || b.mn_major != BMN)
        return TDP_ERR_INVALID_ARG;
    CUtensorMap ta, tb;
    if (!ug_tensor_map(a, AMN ? UG_BK : UG_BM, &ta) || !ug_tensor_map(b, BMN ? UG_BK : BN, &tb))
        return TDP_ERR_INVALID_ARG;
    constexpr size_t smem = (size_t)STAGES * (ug_op_bytes<AMN>(UG_BM) + ug_op_bytes<BMN>(BN)) + EPI::smem_bytes(BN);
    static_assert(smem + 1024 <= 232448, "shared memory");
    auto kern = umma_gemm_kernel<BN, STAGES, AMN, BMN, EPI>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    int kps = (K + splits - 1) / splits;
    kps = (kps + UG_BK - 1) / UG_BK * UG_BK;
    dim3 grid((M + UG_BM - 1) / UG_BM, N / BN, splits);
    kern<<<grid, UG_THREADS, smem, s>>>(ta, tb, epi, K, kps, d_status, spin_limit());
    return cudaGetLastError() == cudaSuccess ? TDP_OK : TDP_ERR_CUDA;
}

// ------------------------------------- pre-pool gradient patches
//
// Rows [base, base + rows) of a pre-pool-gradient patch: row i is dz2 pixel
// (oy, ox) = (i / PITCH - OFF, i % PITCH - OFF) of a cell, 8 channels per
// 16-byte chunk in plane kc (plane_bytes apart, rows 16 bytes apart); rows
// that are no dz2 pixel (padding, dropped columns, past the grid) are zero.
// One work item per (pooled window, 8 channels) loads the pooled gradient
// and the arg-max once and writes the window's four pixels (the value at the
// arg-max pixel, zero at the others).  Items are numbered so that the 8 lanes
// of a 16-byte shared-memory store phase write 8 consecutive windows of one
// plane (rows 2 apart: at most 2-way bank conflicts), and a warp's loads are
// 8 windows x 64 contiguous bytes.  Loading (into registers) and storing are
// separate steps so that the loads can be issued before waiting for the
// destination buffer; a thread holds at most DZ2_ITEMS items.
constexpr int DZ2_ITEMS = 4;

struct Dz2Items {
    uint4 g[DZ2_ITEMS];
    uint2 a[DZ2_ITEMS];
};

template <int PITCH, int OFF>
__device__ __forceinline__ void dz2_window_range(int base, int rows, int &py0, int &nwin)
{
    const int oy0 = max(0, base / PITCH - OFF), oy1 = min(C2 - 1, (base + rows - 1) / PITCH - OFF);
    py0 = oy0 >> 1;
    nwin = oy1 < oy0 ? 0 : ((oy1 >> 1) - py0 + 1) * PO;
}

__device__ __forceinline__ void dz2_item(int c, int &w, int &kc)
{
    w = ((c >> 6) << 3) | (c & 7);
    kc = ((c >> 3) & 3) | (((c >> 5) & 1) << 2);
}

template <int PITCH, int OFF>
__device__ __forceinline__ void dz2_load(Dz2Items &it, int base, int rows, const bf16 *__restrict__ dy2p,
                                         const uint8_t *__restrict__ argmax, long long cell, int tid, int nthreads)
{
    int py0, nwin;
    dz2_window_range<PITCH, OFF>(base, rows, py0, nwin);
    const int nitems = ((nwin + 7) >> 3) << 6;
#pragma unroll
    for (int k = 0; k < DZ2_ITEMS; k++) {
        const int c = tid + k * nthreads;
        int w, kc;
        dz2_item(c, w, kc);
        if (c < nitems && w < nwin) {
            const size_t q = ((size_t)cell * PO + py0 + w / PO) * PO + w % PO;
            it.g[k] = __ldg((const uint4 *)(dy2p + q * CH2 + kc * 8));
            it.a[k] = __ldg((const uint2 *)(argmax + q * CH2 + kc * 8));
        }
    }
}

template <int PITCH, int OFF>
__device__ __forceinline__ void dz2_store(const Dz2Items &it, unsigned char *planes, int plane_bytes, int base,
                                          int rows, int tid, int nthreads)
{
    // zero rows that hold no dz2 pixel (row-major: a warp writes 32 rows of one plane)
    for (int r = tid; r < rows; r += nthreads) {
        const int i = base + r, oy = i / PITCH - OFF, ox = i % PITCH - OFF;
        if (oy < 0 || oy >= C2 || ox < 0 || ox >= C2)
#pragma unroll
            for (int kc = 0; kc < 8; kc++)
                *(uint4 *)(planes + kc * plane_bytes + r * 16) = make_uint4(0, 0, 0, 0);
    }
    int py0, nwin;
    dz2_window_range<PITCH, OFF>(base, rows, py0, nwin);
    const int nitems = ((nwin + 7) >> 3) << 6;
#pragma unroll
    for (int k = 0; k < DZ2_ITEMS; k++) {
        const int c = tid + k * nthreads;
        int w, kc;
        dz2_item(c, w, kc);
        if (c >= nitems || w >= nwin)
            continue;
        const int py = py0 + w / PO, px = w % PO;
        const uint32_t gw[4] = {it.g[k].x, it.g[k].y, it.g[k].z, it.g[k].w};
        const uint32_t ab[2] = {it.a[k].x, it.a[k].y};
#pragma unroll
        for (int pos = 0; pos < 4; pos++) {
            const int oy = 2 * py + (pos >> 1), ox = 2 * px + (pos & 1);
            const int r = (oy + OFF) * PITCH + ox + OFF - base;
            if (r < 0 || r >= rows)
                continue;
            uint32_t o[4] = {gw[0], gw[1], gw[2], gw[3]};
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const uint32_t byte = (ab[e >> 2] >> (8 * (e & 3))) & 0xffu;
                if (byte != (uint32_t)pos)
                    o[e >> 1] &= (e & 1) ? 0x0000ffffu : 0xffff0000u;
            }
            *(uint4 *)(planes + kc * plane_bytes + r * 16) = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

// ------------------------------------------ conv2 forward on tcgen05
//
// conv2 + bias + ReLU + 2x2 max-pool on the 5th-gen tensor cores as nine
// accumulating GEMMs, one per tap, over shifted views of one input patch.
// Output pixels of a cell are taken in raster order with the input's row
// pitch of 26 (columns 24 and 25 of each row are computed and discarded), so
// output pixel q' = 26*oy + ox reads input pixel q' + 26*ky + kx for tap
// (ky, kx): the A operand of a tap is the patch seen from a start row moved by
// 26*ky + kx.  A tile is two output row-pairs of one cell (104 useful rows of
// the 128-row MMA); its patch is the 182 input pixels from row 52*t of the
// cell (zero past the cell's 676), stored K-major with one 16-byte core-matrix
// row per (pixel, 8 channels): plane kc (channels 8kc..8kc+7) holds every
// pixel at 16 bytes apart, so an 8-row group is 128 bytes (SBO) and the next
// 8 channels one plane (LBO) further.  W2 of all nine taps stays in shared
// memory for the CTA's whole life (persistent CTAs, tiles in grid-stride
// order).  Per tile: 18 K16 MMAs into a 64-column fp32 accumulator in tensor
// memory; the accumulator then goes through shared memory (a window's four
// rows sit in different warps) for bias + ReLU + the window maximum and its
// first arg-max.  Warp roles: four worker warpgroups, each owning one patch
// stage, one accumulator and one staging buffer, take every fourth tile of
// the CTA (load the patch, hand it to the MMA warp through mbarrier full[g],
// wait for done[g], pool); one more warp issues the MMAs tile by tile.
// Every wait is bounded; a wait that runs out sets TDP_ERR_TIMEOUT in
// d_status.
constexpr int C2_WORKERS = 4;
constexpr int C2_THREADS = 128 * C2_WORKERS + 32;
constexpr int C2_MMA_WARP = 4 * C2_WORKERS;
constexpr int C2_PATCH_ROWS = 192;                  // >= 128 + 2*26 + 2 = 182, whole 8-row groups
constexpr int C2_PLANE = C2_PATCH_ROWS * 16;        // bytes of one 8-channel plane
constexpr int C2_PATCH_BYTES = 4 * C2_PLANE;        // 32 channels
constexpr int C2_W_TAP_BYTES = CH2 * CH1 * 2;       // W2 of one tap, [64 co][32 ci]
constexpr int C2_W_BYTES = 9 * C2_W_TAP_BYTES;
constexpr int C2_ACC_PITCH = CH2 + 4;               // floats per staged accumulator row
constexpr int C2_ACC_BYTES = 128 * C2_ACC_PITCH * 4; // the accumulator staged for the pool
constexpr int C2_STAGE_BYTES = C2_PATCH_BYTES + C2_ACC_BYTES;
constexpr int C2_TILES_PER_CELL = C2 / 4;           // 6 tiles of 2 row-pairs
constexpr uint32_t C2_TMEM_COLS = 64;               // one accumulator
constexpr uint32_t C2_TMEM_ALLOC = C2_WORKERS * C2_TMEM_COLS;
static_assert(C2_W_BYTES + C2_WORKERS * C2_STAGE_BYTES + 1024 <= 232448, "conv2 forward shared memory");

// Barrier among the 128 threads of warpgroup g (ids 1.. ; 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int g)
{
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}

// The same barrier with an OR over the threads' flags: every thread of the
// warpgroup gets the same answer (so they leave a loop together).
__device__ __forceinline__ bool wg_any(int g, bool flag)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)flag), "r"(g + 1)
                 : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(C2_THREADS) conv2_pool_umma_kernel(const bf16 *__restrict__ y1,
                                                                     const bf16 *__restrict__ w2,
                                                                     const float *__restrict__ bias, bf16 *y2,
                                                                     uint8_t *argmax, long long ntiles,
                                                                     int32_t *d_status, uint32_t limit)
{
    extern __shared__ __align__(1024) unsigned char c2_smem[];
    unsigned char *sw = c2_smem;              // W2, 9 taps
    unsigned char *sst = c2_smem + C2_W_BYTES; // per worker: patch, then staged accumulator
    __shared__ __align__(8) uint64_t s_full[C2_WORKERS], s_done[C2_WORKERS], s_fin;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    __shared__ __align__(16) float s_bias[CH2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(128, CH2);

    if (tid < CH2)
        s_bias[tid] = bias[tid];
    if (tid == 0) {
        for (int g = 0; g < C2_WORKERS; g++) {
            mbar_init(&s_full[g], 128);
            mbar_init(&s_done[g], 1);
        }
        mbar_init(&s_fin, 1);
        s_err = 0;
    }
    if (warp == C2_MMA_WARP) {
        umma::tmem_alloc(&s_tmem, C2_TMEM_ALLOC);
        umma::fence_before_sync();
    }
    // W2 [co][ky][kx][ci] -> tap t = ky*3 + kx: K-major [co][ci] core matrices
    for (int c = tid; c < 9 * CH2 * 4; c += C2_THREADS) {
        const int t = c / (CH2 * 4), co = (c / 4) % CH2, kc = c % 4;
        cnn::cp_async16(sw + t * C2_W_TAP_BYTES + umma::chunk_off(co, kc, 4), w2 + ((size_t)co * 9 + t) * CH1 + kc * 8,
                        true);
    }
    cnn::cp_async_commit();
    cnn::cp_async_wait<0>();
    fence_proxy_async_smem(); // W2 visible to the tensor cores
    __syncthreads();          // ... and the mbarriers, tensor-memory address and bias
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp < C2_MMA_WARP) {
        // worker warpgroup g: the CTA's tiles g, g + 4, ...
        const int g = warp >> 2, ptid = tid & 127, q = warp & 3;
        unsigned char *patch = sst + g * C2_STAGE_BYTES;
        float *sacc = (float *)(patch + C2_PATCH_BYTES);
        const uint32_t acc = tmem + (uint32_t)(g * C2_TMEM_COLS) + ((uint32_t)(32 * q) << 16);
        uint32_t dphase = 0;
        for (long long it = g; it < my_tiles; it += C2_WORKERS) {
            const long long tile = blockIdx.x + it * gridDim.x;
            const long long cell = tile / C2_TILES_PER_CELL;
            const int t = (int)(tile % C2_TILES_PER_CELL);
            // the patch: pixel 104t + r (r < 192) of the cell, 8 channels per 16-byte chunk
            // (its last reader, this warpgroup's previous tile's MMAs, has completed)
            const bf16 *src = y1 + (size_t)cell * C1 * C1 * CH1;
            for (int c = ptid; c < C2_PATCH_ROWS * 4; c += 128) {
                const int r = c >> 2, kc = c & 3, pix = 4 * C1 * t + r;
                const bool in = pix < C1 * C1;
                cnn::cp_async16(patch + kc * C2_PLANE + r * 16, in ? src + (size_t)pix * CH1 + kc * 8 : nullptr,
                                in);
            }
            cnn::cp_async_commit();
            cnn::cp_async_wait<0>();
            fence_proxy_async_smem();
            umma::fence_before_sync();
            mbar_arrive(&s_full[g]);
            const bool done = mbar_wait(&s_done[g], dphase, limit);
            if (wg_any(g, !done)) { // the warpgroup leaves together (its barriers below)
                s_err = 1;
                break;
            }
            dphase ^= 1u;
            umma::fence_after_sync();
            // accumulator rows (TMEM lane = row) to shared memory: warp q takes
            // lanes 32q.., all 64 columns (row pitch C2_ACC_PITCH: the lanes'
            // 16-byte stores hit distinct banks)
#pragma unroll 1
            for (int cb = 0; cb < CH2; cb += 16) {
                float v[16];
                umma::ld_16cols(acc + cb, v);
                float4 *dst = (float4 *)(sacc + (32 * q + lane) * C2_ACC_PITCH + cb);
#pragma unroll
                for (int e = 0; e < 4; e++)
                    dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
            }
            wg_sync(g); // accumulator staged
            // pool: 2 row-pairs x 12 windows x 16 groups of 4 channels (lanes read
            // consecutive 16-byte chunks); window (P, px) = rows 52P + 2px +
            // {0, 1, 26, 27}, (dy, dx) = (0,0) (0,1) (1,0) (1,1)
            for (int o = ptid; o < 2 * PO * (CH2 / 4); o += 128) {
                const int cg = o % (CH2 / 4), w = o / (CH2 / 4), P = w / PO, px = w % PO;
                const int r0 = 52 * P + 2 * px;
                const int rows[4] = {r0, r0 + 1, r0 + C1, r0 + C1 + 1};
                const float4 bb = *(const float4 *)(s_bias + cg * 4);
                float best[4];
                int arg[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float4 a = *(const float4 *)(sacc + rows[e] * C2_ACC_PITCH + cg * 4);
                    const float x[4] = {fmaxf(a.x + bb.x, 0.f), fmaxf(a.y + bb.y, 0.f), fmaxf(a.z + bb.z, 0.f),
                                        fmaxf(a.w + bb.w, 0.f)};
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (e == 0 || x[c] > best[c]) { // first maximum wins
                            best[c] = x[c];
                            arg[c] = e;
                        }
                }
                __align__(8) bf16 ov[4];
                __align__(4) uint8_t oa[4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    ov[c] = __float2bfloat16_rn(best[c]);
                    oa[c] = (uint8_t)arg[c];
                }
                const size_t qo = ((size_t)cell * PO + 2 * t + P) * PO + px; // pooled pixel (cell, py, px)
                *(uint2 *)(y2 + qo * CH2 + cg * 4) = *(const uint2 *)ov;
                *(uint32_t *)(argmax + qo * CH2 + cg * 4) = *(const uint32_t *)oa;
            }
            wg_sync(g); // the staged accumulator is read
        }
    } else {
        // the MMA warp: tiles in order, stage and accumulator it % 4; one elected lane issues
        for (long long it = 0; it < my_tiles; it++) {
            const int g = (int)(it % C2_WORKERS);
            if (!__all_sync(0xffffffffu, mbar_wait(&s_full[g], (uint32_t)(it / C2_WORKERS) & 1u, limit))) {
                s_err = 1;
                break;
            }
            umma::fence_after_sync();
            // descriptors differ only in their start address (16-byte units, low bits)
            const uint64_t da = umma::smem_desc(smem_addr(sst + g * C2_STAGE_BYTES), C2_PLANE, 128);
            const uint64_t db = umma::smem_desc(smem_addr(sw), 128, 512);
            const uint32_t d = tmem + (uint32_t)(g * C2_TMEM_COLS);
            if (umma::elect_one()) {
#pragma unroll
                for (int tap = 0; tap < 9; tap++) {
                    const uint32_t shift = (uint32_t)((tap / 3) * C1 + tap % 3); // start row 26*ky + kx
#pragma unroll
                    for (int j = 0; j < 2; j++) // channels 16j..16j+15: planes 2j, 2j+1
                        umma::mma_bf16(d, da + shift + 2 * j * (C2_PLANE / 16),
                                       db + (uint32_t)(tap * C2_W_TAP_BYTES + j * 256) / 16, idesc,
                                       tap > 0 || j > 0);
                }
                umma::commit(&s_done[g]);
            }
            __syncwarp();
        }
        if (umma::elect_one())
            umma::commit(&s_fin); // arrives once every MMA issued above has completed
        __syncwarp();
        if (!__all_sync(0xffffffffu, mbar_wait(&s_fin, 0, limit)))
            s_err = 1;
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_err)
        set_status(d_status, TDP_ERR_TIMEOUT);
    if (warp == C2_MMA_WARP) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, C2_TMEM_ALLOC);
    }
}

// ------------------------------------ conv2 data gradient on tcgen05
//
// dz1[cell][y][x][ci] = (y1 > 0) * sum_{ky,kx,co} dz2[cell][y-ky][x-kx][co]
// W2[co][ky][kx][ci], dz2 the pre-pool gradient (the pooled gradient at its
// window's arg-max pixel, 0 elsewhere; zero outside the 24x24 output).  As in
// the forward, nine accumulating GEMMs over shifted views of one patch:
// input pixels are taken in raster order with pitch 28 over a zero-padded
// 28 x 28 grid dzp (dzp[a][b] = dz2[a-2][b-2]), so pixel m' = 28y + x reads
// dzp[m' + 28(2-ky) + (2-kx)] for tap (ky, kx); columns 26, 27 are dropped.
// A tile is 128 consecutive m' of one cell (6 tiles per cell, the last
// partial); its patch is dzp[128t .. 128t + 191], computed from the pooled
// gradient and the arg-max (8 channels per 16-byte chunk) straight into 8
// K-major planes.  W2 of every tap is kept transposed as [32 ci][64 co]
// core matrices for the CTA's life.  N = 32 (ci), 4 K16 steps per tap.  The
// epilogue applies the ReLU mask of y1 from registers (no shared memory).
// Warp roles: four worker warpgroups, each owning one patch stage and one
// 32-column accumulator, take every fourth tile of the CTA: build the patch,
// hand it to the MMA warp (mbarrier full[g], 128 arrivals), fetch the next
// tile's pooled gradient, wait for the MMAs (done[g], tcgen05.commit) and
// write the masked dz1 rows; one more warp issues the MMAs tile by tile.
// While one warpgroup waits on memory the others build, drain or compute.
constexpr int DG_WORKERS = 4;
constexpr int DG_THREADS = 128 * DG_WORKERS + 32;
constexpr int DG_MMA_WARP = 4 * DG_WORKERS;
constexpr int DG_P = 28;                              // padded pitch
constexpr int DG_PIX = C1 * DG_P;                     // m' per cell: 26 rows x 28
constexpr int DG_TILES_PER_CELL = (DG_PIX + 127) / 128; // 6
constexpr int DG_PATCH_ROWS = 192;                    // >= 128 + 2*28 + 2 = 186
constexpr int DG_PLANE = DG_PATCH_ROWS * 16;
constexpr int DG_PATCH_BYTES = 8 * DG_PLANE;          // 64 channels
constexpr int DG_W_TAP_BYTES = CH1 * CH2 * 2;         // [32 ci][64 co]
constexpr int DG_W_BYTES = 9 * DG_W_TAP_BYTES;
constexpr uint32_t DG_TMEM_COLS = 32;                 // one accumulator
constexpr uint32_t DG_TMEM_ALLOC = DG_WORKERS * DG_TMEM_COLS;
static_assert(DG_W_BYTES + DG_WORKERS * DG_PATCH_BYTES + 1024 <= 232448, "conv2 data gradient shared memory");

__global__ void __launch_bounds__(DG_THREADS) conv2_dgrad_umma_kernel(const bf16 *__restrict__ dy2p,
                                                                      const uint8_t *__restrict__ argmax,
                                                                      const bf16 *__restrict__ w2,
                                                                      const bf16 *__restrict__ y1, bf16 *dz1,
                                                                      long long ntiles, int32_t *d_status,
                                                                      uint32_t limit)
{
    extern __shared__ __align__(1024) unsigned char dg_smem[];
    unsigned char *sw = dg_smem;              // W2 transposed, 9 taps
    unsigned char *sp = dg_smem + DG_W_BYTES; // one patch per worker warpgroup
    __shared__ __align__(8) uint64_t s_full[DG_WORKERS], s_done[DG_WORKERS], s_fin;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(128, CH1);

    if (tid == 0) {
        for (int g = 0; g < DG_WORKERS; g++) {
            mbar_init(&s_full[g], 128);
            mbar_init(&s_done[g], 1);
        }
        mbar_init(&s_fin, 1);
        s_err = 0;
    }
    if (warp == DG_MMA_WARP) {
        umma::tmem_alloc(&s_tmem, DG_TMEM_ALLOC);
        umma::fence_before_sync();
    }
    // W2[co][tap][ci] -> tap: K-major [ci][co]: chunk (ci, kc) = co 8kc..8kc+7
    for (int c = tid; c < 9 * CH1 * (CH2 / 8); c += DG_THREADS) {
        const int tap = c / (CH1 * 8), ci = (c / 8) % CH1, kc = c % 8;
        __align__(16) bf16 v[8];
#pragma unroll
        for (int e = 0; e < 8; e++)
            v[e] = w2[((size_t)(kc * 8 + e) * 9 + tap) * CH1 + ci];
        *(uint4 *)(sw + tap * DG_W_TAP_BYTES + umma::chunk_off(ci, kc, 8)) = *(const uint4 *)v;
    }
    fence_proxy_async_smem(); // W2 visible to the tensor cores
    __syncthreads();          // ... and the mbarriers and tensor-memory address
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp < DG_MMA_WARP) {
        // worker warpgroup g: the CTA's tiles g, g + 4, ... (patch stage g, accumulator g)
        const int g = warp >> 2, ptid = tid & 127, q = warp & 3;
        unsigned char *stage = sp + g * DG_PATCH_BYTES;
        const uint32_t acc = tmem + (uint32_t)(g * DG_TMEM_COLS) + ((uint32_t)(32 * q) << 16);
        uint32_t dphase = 0;
        Dz2Items items;
        if (g < my_tiles) {
            const long long tile = blockIdx.x + (long long)g * gridDim.x;
            dz2_load<DG_P, 2>(items, (int)(tile % DG_TILES_PER_CELL) * 128, DG_PATCH_ROWS, dy2p, argmax,
                              tile / DG_TILES_PER_CELL, ptid, 128);
        }
        for (long long it = g; it < my_tiles; it += DG_WORKERS) {
            const long long tile = blockIdx.x + it * gridDim.x;
            const long long cell = tile / DG_TILES_PER_CELL;
            const int i0 = (int)(tile % DG_TILES_PER_CELL) * 128;
            // the stage's last reader, this warpgroup's previous tile's MMAs, has completed
            dz2_store<DG_P, 2>(items, stage, DG_PLANE, i0, DG_PATCH_ROWS, ptid, 128);
            fence_proxy_async_smem();
            umma::fence_before_sync(); // the previous tile's accumulator loads precede the hand-over
            mbar_arrive(&s_full[g]);
            if (it + DG_WORKERS < my_tiles) { // the next tile's pooled gradient, in flight meanwhile
                const long long nt = tile + (long long)DG_WORKERS * gridDim.x;
                dz2_load<DG_P, 2>(items, (int)(nt % DG_TILES_PER_CELL) * 128, DG_PATCH_ROWS, dy2p, argmax,
                                  nt / DG_TILES_PER_CELL, ptid, 128);
            }
            if (!mbar_wait(&s_done[g], dphase, limit)) {
                s_err = 1;
                break;
            }
            dphase ^= 1u;
            umma::fence_after_sync();
            // epilogue: warp q holds m' = i0 + 32q + lane, all 32 ci
            float v0[16], v1[16];
            umma::ld_16cols(acc, v0);
            umma::ld_16cols(acc + 16, v1);
            const int i = i0 + 32 * q + lane, y = i / DG_P, x = i % DG_P;
            if (i < DG_PIX && x < C1) {
                const size_t o = (((size_t)cell * C1 + y) * C1 + x) * CH1;
                const uint4 *mk = (const uint4 *)(y1 + o);
                uint4 mm[4];
#pragma unroll
                for (int h = 0; h < 4; h++)
                    mm[h] = mk[h];
                uint4 *dst = (uint4 *)(dz1 + o);
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const bf16 *mb = (const bf16 *)&mm[h];
                    __align__(16) bf16 ov[8];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const float val = h < 2 ? v0[8 * h + e] : v1[8 * (h - 2) + e];
                        ov[e] = __float2bfloat16_rn(bf2f(mb[e]) > 0.f ? val : 0.f);
                    }
                    dst[h] = *(const uint4 *)ov;
                }
            }
        }
    } else {
        // the MMA warp: tiles in order, stage and accumulator it % 4; one elected lane issues
        for (long long it = 0; it < my_tiles; it++) {
            const int g = (int)(it % DG_WORKERS);
            if (!__all_sync(0xffffffffu, mbar_wait(&s_full[g], (uint32_t)(it / DG_WORKERS) & 1u, limit))) {
                s_err = 1;
                break;
            }
            umma::fence_after_sync();
            // descriptors differ only in their start address (16-byte units, low bits)
            const uint64_t da = umma::smem_desc(smem_addr(sp + g * DG_PATCH_BYTES), DG_PLANE, 128);
            const uint64_t db = umma::smem_desc(smem_addr(sw), 128, 1024);
            const uint32_t d = tmem + (uint32_t)(g * DG_TMEM_COLS);
            if (umma::elect_one()) {
#pragma unroll
                for (int tap = 0; tap < 9; tap++) {
                    const int ky = tap / 3, kx = tap % 3;
                    const uint32_t shift = (uint32_t)((2 - ky) * DG_P + (2 - kx));
#pragma unroll
                    for (int j = 0; j < CH2 / 16; j++) // co 16j..16j+15: planes 2j, 2j+1
                        umma::mma_bf16(d, da + shift + 2 * j * (DG_PLANE / 16),
                                       db + (uint32_t)(tap * DG_W_TAP_BYTES + j * 256) / 16, idesc,
                                       tap > 0 || j > 0);
                }
                umma::commit(&s_done[g]);
            }
            __syncwarp();
        }
        if (umma::elect_one())
            umma::commit(&s_fin); // arrives once every MMA issued above has completed
        __syncwarp();
        if (!__all_sync(0xffffffffu, mbar_wait(&s_fin, 0, limit)))
            s_err = 1;
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_err)
        set_status(d_status, TDP_ERR_TIMEOUT);
    if (warp == DG_MMA_WARP) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, DG_TMEM_ALLOC);
    }
}

// ---------------------------------- conv2 weight gradient on tcgen05
//
// dW[co][tap][ci] = sum_p dz2[p][co] y1[p + shift(tap)][ci] over every output
// pixel p of every cell, as nine accumulating GEMMs per tile of pixels with
// the pixels as K: output pixels in raster order with pitch 26 (p' = 26 oy +
// ox; dz2 is 0 for ox >= 24, so the padding adds nothing) make tap (ky, kx)
// the input patch shifted by 26 ky + kx rows.  Both operands are MN-major
// (the channel dimension contiguous in 16-byte rows of 8 channels, one row
// per pixel): A = dz2 of the tile's 128 pixels in 8 planes of 8 co (built
// from the pooled gradient and the arg-max), B = y1 of its 182 input pixels
// in 4 planes of 8 ci (cp.async).  M = 64 (co; TMEM lane 32(co/16) + co%16),
// N = 32 (ci), one 32-column accumulator per tap (288 of 512 columns).  A
// persistent CTA accumulates its tiles in tensor memory and writes one fp32
// partial of dW at the end; the partials are summed in block order (fixed).
// Warp roles: four producer warpgroups each own one stage and build every
// fourth tile of the CTA (so four tiles' load latencies overlap); one more
// warp allocates tensor memory and issues the MMAs, tile by tile in order.
// Stage s is handed over by mbarriers: full[s] (128 producer arrivals after
// the patches are written) and empty[s] (tcgen05.commit once the MMAs that
// read it have completed).
constexpr int WG_PRODUCERS = 4;                         // warpgroups = stages
constexpr int WG_THREADS = 128 * WG_PRODUCERS + 32;     // + the MMA warp
constexpr int WG_MMA_WARP = 4 * WG_PRODUCERS;
constexpr int WG_PIX = C2 * C1;                        // p' per cell: 24 rows x 26
constexpr int WG_TILES_PER_CELL = (WG_PIX + 127) / 128; // 5
constexpr int WG_A_PLANE = 128 * 16;
constexpr int WG_A_BYTES = 8 * WG_A_PLANE;              // 64 co
constexpr int WG_B_ROWS = 192;                          // >= 128 + 2*26 + 2 = 182
constexpr int WG_B_PLANE = WG_B_ROWS * 16;
constexpr int WG_B_BYTES = 4 * WG_B_PLANE;              // 32 ci
constexpr int WG_BUF_BYTES = WG_A_BYTES + WG_B_BYTES;
constexpr uint32_t WG_TMEM_COLS = 512;

__global__ void __launch_bounds__(WG_THREADS) conv2_wgrad_umma_kernel(const bf16 *__restrict__ dy2p,
                                                                      const uint8_t *__restrict__ argmax,
                                                                      const bf16 *__restrict__ y1, long long ntiles,
                                                                      float *__restrict__ part, int32_t *d_status,
                                                                      uint32_t limit)
{
    extern __shared__ __align__(1024) unsigned char wg_smem[]; // one stage per producer: A patch, then B patch
    __shared__ __align__(8) uint64_t s_full[WG_PRODUCERS], s_empty[WG_PRODUCERS], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // M = 64, N = 32, both operands MN-major (bits 15, 16)
    constexpr uint32_t idesc = umma::idesc_bf16_f32(64, CH1) | (1u << 15) | (1u << 16);

    if (tid == 0) {
        for (int g = 0; g < WG_PRODUCERS; g++) {
            mbar_init(&s_full[g], 128);
            mbar_init(&s_empty[g], 1);
        }
        mbar_init(&s_done, 1);
        s_err = 0;
    }
    if (warp == WG_MMA_WARP) {
        umma::tmem_alloc(&s_tmem, WG_TMEM_COLS);
        umma::fence_before_sync();
    }
    __syncthreads(); // the mbarriers and the tensor-memory address
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp < WG_MMA_WARP) {
        // producer warpgroup g: the CTA's tiles g, g + 4, ... into stage g
        const int g = warp >> 2, ptid = tid & 127;
        unsigned char *a = wg_smem + g * WG_BUF_BYTES, *b = a + WG_A_BYTES;
        uint32_t ephase = 0;
        for (long long it = g; it < my_tiles; it += WG_PRODUCERS) {
            const long long tile = blockIdx.x + it * gridDim.x;
            const long long cell = tile / WG_TILES_PER_CELL;
            const int i0 = (int)(tile % WG_TILES_PER_CELL) * 128;
            // the pooled gradient and arg-max of the tile, in flight during the wait
            Dz2Items items;
            dz2_load<C1, 0>(items, i0, 128, dy2p, argmax, cell, ptid, 128);
            if (it >= WG_PRODUCERS) { // the MMAs of tile it - 4 have read the stage
                if (!mbar_wait(&s_empty[g], ephase, limit)) {
                    s_err = 1;
                    break;
                }
                ephase ^= 1u;
            }
            // B: input pixels i0 + r (r < 192) of the cell, 8 ci per chunk (cp.async)
            const bf16 *src = y1 + (size_t)cell * C1 * C1 * CH1;
            for (int c = ptid; c < WG_B_ROWS * 4; c += 128) {
                const int r = c >> 2, kc = c & 3, pix = i0 + r;
                const bool in = pix < C1 * C1;
                cnn::cp_async16(b + kc * WG_B_PLANE + r * 16, in ? src + (size_t)pix * CH1 + kc * 8 : nullptr, in);
            }
            cnn::cp_async_commit();
            // A: dz2 at output pixels p' = i0 + r (r < 128), 8 co per chunk
            dz2_store<C1, 0>(items, a, WG_A_PLANE, i0, 128, ptid, 128);
            cnn::cp_async_wait<0>();
            fence_proxy_async_smem(); // this thread's patch writes, visible to the tensor cores
            mbar_arrive(&s_full[g]);
        }
    } else {
        // the MMA warp: tiles in order, stage it % 4; warp-uniform descriptors, one elected lane issues
        for (long long it = 0; it < my_tiles; it++) {
            const int st = (int)(it % WG_PRODUCERS);
            if (!__all_sync(0xffffffffu, mbar_wait(&s_full[st], (uint32_t)(it / WG_PRODUCERS) & 1u, limit))) {
                s_err = 1;
                break;
            }
            umma::fence_after_sync();
            // descriptors differ only in their start address (16-byte units, low bits)
            const uint32_t a = smem_addr(wg_smem + st * WG_BUF_BYTES);
            const uint64_t da = umma::smem_desc(a, 128, WG_A_PLANE),
                           db = umma::smem_desc(a + WG_A_BYTES, 128, WG_B_PLANE);
            if (umma::elect_one()) {
#pragma unroll
                for (int tap = 0; tap < 9; tap++) {
                    const uint32_t shift = (uint32_t)((tap / 3) * C1 + tap % 3); // rows
#pragma unroll
                    for (int j = 0; j < 8; j++) // pixels 16j..16j+15: two 8-row K groups
                        umma::mma_bf16(tmem + (uint32_t)(tap * CH1), da + 16 * j, db + shift + 16 * j, idesc,
                                       it > 0 || j > 0);
                }
                umma::commit(&s_empty[st]);
            }
            __syncwarp();
        }
        if (umma::elect_one())
            umma::commit(&s_done); // arrives once every MMA issued above has completed
        __syncwarp();
    }
    // this CTA's partial of dW: warp w < 4, lanes 0..15 hold co = 16w + lane, columns tap*32 + ci
    if (warp < 4) {
        const bool done = mbar_wait(&s_done, 0, limit);
        umma::fence_after_sync();
        if (!done)
            s_err = 1;
        else if (my_tiles > 0) {
            const int co = 16 * warp + lane;
            float *o = part + (size_t)blockIdx.x * (CH2 * 9 * CH1) + (size_t)co * 9 * CH1;
#pragma unroll 1
            for (int cb = 0; cb < 9 * CH1; cb += 16) {
                float v[16];
                umma::ld_16cols(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
                if (lane < 16) {
                    float4 *d = (float4 *)(o + cb);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_err)
        set_status(d_status, TDP_ERR_TIMEOUT);
    if (warp == WG_MMA_WARP) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, WG_TMEM_COLS);
    }
}

// ---------------------------------------------------------- reductions

// out[i] = act(sum_s part[s][i] + bias[i % ncol]) -> bf16 (ReLU) or f32
__global__ void splitk_reduce_kernel(const float *__restrict__ part, int splits, size_t stride, long long n, int ncol,
                                     const float *__restrict__ bias, int relu, bf16 *out_bf, float *out_f)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float s = 0.f;
    for (int k = 0; k < splits; k++)
        s += part[k * stride + i];
    if (bias)
        s += bias[i % ncol];
    if (relu)
        s = fmaxf(s, 0.f);
    if (out_bf)
        out_bf[i] = __float2bfloat16_rn(s);
    if (out_f)
        out_f[i] = s;
}

// Column sums of a bf16 matrix [rows][C] (C a multiple of 8 dividing 2048,
// rows 16-byte aligned) into fp32 partials [blocks][C].  Thread = 8
// consecutive columns (one 16-byte load, four in flight) of a fixed set of
// rows; the per-thread sums are added in thread order (no atomics: the
// result is reproducible for a given grid).
constexpr int CS_THREADS = 256;

__global__ void __launch_bounds__(CS_THREADS) colsum_bf16_kernel(const bf16 *__restrict__ x, long long rows, int C,
                                                                 float *__restrict__ part)
{
    __shared__ float cs[CS_THREADS * 8];
    const int cv = C / 8, c8 = threadIdx.x % cv, rstep = CS_THREADS / cv;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint4 *xv = (const uint4 *)x;
    auto add = [&](uint4 v) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[2 * j] += __uint_as_float(w[j] << 16);
            acc[2 * j + 1] += __uint_as_float(w[j] & 0xffff0000u);
        }
    };
    if ((int)threadIdx.x < rstep * cv) {
        const long long step = (long long)gridDim.x * rstep;
        long long r = (long long)blockIdx.x * rstep + threadIdx.x / cv;
        for (; r + 3 * step < rows; r += 4 * step) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                v[u] = __ldg(xv + (r + u * step) * cv + c8);
#pragma unroll
            for (int u = 0; u < 4; u++)
                add(v[u]);
        }
        for (; r < rows; r += step)
            add(__ldg(xv + r * cv + c8));
    }
#pragma unroll
    for (int j = 0; j < 8; j++)
        cs[threadIdx.x * 8 + j] = acc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += CS_THREADS) {
        float sum = 0.f;
        for (int q = 0; q < rstep; q++)
            sum += cs[(q * cv + i / 8) * 8 + i % 8];
        part[(size_t)blockIdx.x * C + i] = sum;
    }
}

// Blocks of colsum_bf16_kernel (and partial rows it writes) for rows x C.
static inline int colsum_blocks(long long rows, int C)
{
    const long long rstep = CS_THREADS / (C / 8);
    return (int)std::max<long long>(1, std::min<long long>((rows + rstep - 1) / rstep, 2ll * num_sms()));
}

// out[i] = sum_b part[b * stride + i] in float64, in a fixed order: slice s
// (of PS_SLICES) sums b = s, s + PS_SLICES, ... in order, then the slices are
// added by a fixed tree.  A block covers 32 consecutive outputs.
constexpr int PS_SLICES = 16;

// Output column i goes to out0[i] for i < n0, out1[i - n0] for i < n0 + n1,
// else out2[i - n0 - n1] (the column ranges of one partial row that belong
// to different tensors, reduced in one launch).
struct PsOut {
    float *out0, *out1, *out2;
    int n0, n1;
};

__global__ void __launch_bounds__(32 * PS_SLICES) partial_sum_kernel(const float *__restrict__ part, int nb, int n,
                                                                     size_t stride, PsOut po)
{
    __shared__ double s_acc[PS_SLICES][32];
    const int e = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + e;
    double acc = 0.0;
    if (i < n) {
        int b = sl;
        for (; b + 3 * PS_SLICES < nb; b += 4 * PS_SLICES) {
            const float a0 = part[(size_t)b * stride + i];
            const float a1 = part[(size_t)(b + PS_SLICES) * stride + i];
            const float a2 = part[(size_t)(b + 2 * PS_SLICES) * stride + i];
            const float a3 = part[(size_t)(b + 3 * PS_SLICES) * stride + i];
            acc += a0;
            acc += a1;
            acc += a2;
            acc += a3;
        }
        for (; b < nb; b += PS_SLICES)
            acc += part[(size_t)b * stride + i];
    }
    s_acc[sl][e] = acc;
    __syncthreads();
#pragma unroll
    for (int h = PS_SLICES / 2; h > 0; h >>= 1) {
        if (sl < h)
            s_acc[sl][e] += s_acc[sl + h][e];
        __syncthreads();
    }
    if (sl == 0 && i < n) {
        const float r = (float)s_acc[0][e];
        if (i < po.n0)
            po.out0[i] = r;
        else if (i < po.n0 + po.n1)
            po.out1[i - po.n0] = r;
        else
            po.out2[i - po.n0 - po.n1] = r;
    }
}

static inline PsOut ps_out(float *o) { return PsOut{o, nullptr, nullptr, 1 << 30, 0}; }

static inline unsigned psum_blocks(int n) { return (unsigned)((n + 31) / 32); }

// conv1 weight and bias gradients, dW1[co][ky][kx] = sum x0[oy+ky][ox+kx] *
// dz1[oy][ox][co] and db1[co] = sum dz1[..][co] over all cells.  Thread
// (cp, g) owns channels 2cp, 2cp+1 and output rows g, g+13 of every cell of
// its block: one 4-byte load of dz1 feeds 20 accumulators (nine taps and the
// bias for both channels), with the 3x3 image window sliding along the row
// in registers.  The next cell's image is fetched while this one is reduced.
// Per-block partials: the 13 row groups are added in a fixed order.
constexpr int W1_ROWG = C1 / 2;                // 13 row groups of two rows
constexpr int W1_THREADS = 16 * (W1_ROWG + 1); // 224 = 7 warps; group 13 only fetches images
constexpr int W1_BLOCKS_PER_SM = 3;
constexpr int W1_FETCH = (CELL * CELL + W1_THREADS - 1) / W1_THREADS; // image bytes per thread

__global__ void __launch_bounds__(W1_THREADS, W1_BLOCKS_PER_SM)
    conv1_wgrad_kernel(const bf16 *__restrict__ dz1, const uint8_t *__restrict__ grids, long long ncell,
                       long long cells_per_block, float *__restrict__ part)
{
    __shared__ float simg[2][CELL * CELL];
    __shared__ float sred[W1_ROWG][CH1 * 10];
    const int tid = threadIdx.x, cp = tid % 16, g = tid / 16;
    const long long c0 = (long long)blockIdx.x * cells_per_block, c1 = min(ncell, c0 + cells_per_block);
    float acc[2][10];
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
        for (int t = 0; t < 10; t++)
            acc[j][t] = 0.f;
    uint8_t pre[W1_FETCH];
    auto fetch = [&](long long c) {
        const long long gi = c / CELLS_PER_GRID;
        const int r = (int)(c % CELLS_PER_GRID) / GRID_W, cc = (int)(c % GRID_W);
        const uint8_t *img = grids + gi * (GRID_H * CELL) * (GRID_W * CELL) +
                             (long long)(r * CELL) * (GRID_W * CELL) + cc * CELL;
#pragma unroll
        for (int k = 0; k < W1_FETCH; k++) {
            const int i = tid + k * W1_THREADS;
            if (i < CELL * CELL)
                pre[k] = img[(i / CELL) * (GRID_W * CELL) + i % CELL];
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int k = 0; k < W1_FETCH; k++) {
            const int i = tid + k * W1_THREADS;
            if (i < CELL * CELL)
                simg[buf][i] = (float)pre[k] * (1.0f / 255.0f);
        }
    };
    if (c0 < c1) {
        fetch(c0);
        store(0);
    }
    for (long long c = c0; c < c1; c++) {
        const int buf = (int)((c - c0) & 1);
        __syncthreads(); // simg[buf] is written; simg[buf ^ 1] is no longer read
        if (c + 1 < c1)
            fetch(c + 1);
        if (g < W1_ROWG) {
#pragma unroll 1
            for (int h = 0; h < 2; h++) {
                const int oy = g + W1_ROWG * h;
                // the row's 26 channel pairs loaded before any is used
                const uint32_t *drow = (const uint32_t *)(dz1 + (c * C1 + oy) * (C1 * CH1)) + cp;
                uint32_t dv[C1];
#pragma unroll
                for (int ox = 0; ox < C1; ox++)
                    dv[ox] = __ldg(drow + ox * (CH1 / 2));
                const float *row = simg[buf] + oy * CELL;
                float w[3][3];
#pragma unroll
                for (int ky = 0; ky < 3; ky++) {
                    w[ky][0] = row[ky * CELL];
                    w[ky][1] = row[ky * CELL + 1];
                }
#pragma unroll
                for (int ox = 0; ox < C1; ox++) {
#pragma unroll
                    for (int ky = 0; ky < 3; ky++)
                        w[ky][2] = row[ky * CELL + ox + 2];
                    // bf16 pair: channel 2cp in the low half, 2cp+1 in the high half
                    const float d0 = __uint_as_float(dv[ox] << 16), d1 = __uint_as_float(dv[ox] & 0xffff0000u);
#pragma unroll
                    for (int ky = 0; ky < 3; ky++)
#pragma unroll
                        for (int kx = 0; kx < 3; kx++) {
                            acc[0][ky * 3 + kx] = fmaf(d0, w[ky][kx], acc[0][ky * 3 + kx]);
                            acc[1][ky * 3 + kx] = fmaf(d1, w[ky][kx], acc[1][ky * 3 + kx]);
                        }
                    acc[0][9] += d0;
                    acc[1][9] += d1;
#pragma unroll
                    for (int ky = 0; ky < 3; ky++) {
                        w[ky][0] = w[ky][1];
                        w[ky][1] = w[ky][2];
                    }
                }
            }
        }
        if (c + 1 < c1)
            store(buf ^ 1);
    }
    if (g < W1_ROWG) {
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int co = 2 * cp + j;
#pragma unroll
            for (int t = 0; t < 9; t++)
                sred[g][co * 9 + t] = acc[j][t];
            sred[g][CH1 * 9 + co] = acc[j][9];
        }
    }
    __syncthreads();
    // each partial row: 288 weight sums (co-major), then the 32 bias sums
    for (int i = tid; i < CH1 * 10; i += W1_THREADS) {
        float sum = 0.f;
        for (int gg = 0; gg < W1_ROWG; gg++)
            sum += sred[gg][i];
        part[(size_t)blockIdx.x * (CH1 * 10) + i] = sum;
    }
}

// ------------------------------------------------------------------- head
//
// One block per grid: fc2 + softmax (the PE column), the soft query
// cnt[k] = sum_c P[c][k], rsum[r] = sum_{c in row r} sum_k k P[c][k], and,
// when targets are given, the MSE loss and its backward down to dh1 plus the
// fc2 gradients (per-grid partials, summed later in a fixed order).
constexpr int HEAD_THREADS = 256;
constexpr int NPRED = NCLS + GRID_H;

__global__ void __launch_bounds__(HEAD_THREADS) head_kernel(const bf16 *__restrict__ h1, long long ngrid,
                                                            const float *__restrict__ w, const float *__restrict__ b,
                                                            const float *__restrict__ target, float inv_nout,
                                                            float *__restrict__ logits_out, float *__restrict__ P_out,
                                                            float *__restrict__ pred_out, bf16 *__restrict__ dh1,
                                                            float *__restrict__ part)
{
    __shared__ float sh[CELLS_PER_GRID][HID];
    __shared__ float sw[NCLS][HID];
    __shared__ float sP[CELLS_PER_GRID][NCLS];
    __shared__ float sdl[CELLS_PER_GRID][NCLS];
    __shared__ float spred[NPRED], sdpred[NPRED];
    const long long grid = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < CELLS_PER_GRID * HID; i += HEAD_THREADS)
        sh[i / HID][i % HID] = bf2f(h1[grid * CELLS_PER_GRID * HID + i]);
    for (int i = tid; i < NCLS * HID; i += HEAD_THREADS)
        sw[i / HID][i % HID] = w[i];
    __syncthreads();
    if (tid < CELLS_PER_GRID * NCLS) {
        int c = tid / NCLS, k = tid % NCLS;
        float s = b[k];
        for (int u = 0; u < HID; u++)
            s = fmaf(sh[c][u], sw[k][u], s);
        sP[c][k] = s;
        if (logits_out)
            logits_out[(grid * CELLS_PER_GRID + c) * NCLS + k] = s;
    }
    __syncthreads();
    if (tid < CELLS_PER_GRID) {
        float mx = sP[tid][0];
        for (int k = 1; k < NCLS; k++)
            mx = fmaxf(mx, sP[tid][k]);
        float e[NCLS], z = 0.f;
        for (int k = 0; k < NCLS; k++) {
            e[k] = expf(sP[tid][k] - mx);
            z += e[k];
        }
        float iz = 1.0f / z;
        for (int k = 0; k < NCLS; k++)
            sP[tid][k] = e[k] * iz;
    }
    __syncthreads();
    if (P_out && tid < CELLS_PER_GRID * NCLS)
        P_out[grid * CELLS_PER_GRID * NCLS + tid] = sP[tid / NCLS][tid % NCLS];
    if (tid < NPRED) {
        float s = 0.f;
        if (tid < NCLS) {
            for (int c = 0; c < CELLS_PER_GRID; c++)
                s += sP[c][tid];
        } else {
            int r = tid - NCLS;
            for (int c = r * GRID_W; c < r * GRID_W + GRID_W; c++)
                for (int k = 0; k < NCLS; k++)
                    s = fmaf((float)k, sP[c][k], s);
        }
        spred[tid] = s;
        if (pred_out)
            pred_out[grid * NPRED + tid] = s;
        if (target) {
            float d = s - target[grid * NPRED + tid];
            sdpred[tid] = 2.f * d * inv_nout;
        }
    }
    if (!target)
        return;
    __syncthreads();
    float *gp = part + grid * (NCLS * HID + NCLS + 1);
    if (tid == 0) {
        float l = 0.f;
        for (int j = 0; j < NPRED; j++) {
            float d = spred[j] - target[grid * NPRED + j];
            l += d * d;
        }
        gp[NCLS * HID + NCLS] = l * inv_nout; // the grid's share of the mean

    }
    if (tid < CELLS_PER_GRID) {
        const int c = tid, r = c / GRID_W;
        float dP[NCLS], dot = 0.f;
        for (int k = 0; k < NCLS; k++) {
            dP[k] = sdpred[k] + (float)k * sdpred[NCLS + r];
            dot = fmaf(sP[c][k], dP[k], dot);
        }
        for (int k = 0; k < NCLS; k++)
            sdl[c][k] = sP[c][k] * (dP[k] - dot);
    }
    __syncthreads();
    // dh1[c][u] = (sum_k dl[c][k] w[k][u]) * (h1 > 0)
    for (int i = tid; i < CELLS_PER_GRID * HID; i += HEAD_THREADS) {
        int c = i / HID, u = i % HID;
        float s = 0.f;
        for (int k = 0; k < NCLS; k++)
            s = fmaf(sdl[c][k], sw[k][u], s);
        dh1[grid * CELLS_PER_GRID * HID + i] = __float2bfloat16_rn(sh[c][u] > 0.f ? s : 0.f);
    }
    // fc2 gradient partials of this grid
    for (int i = tid; i < NCLS * HID; i += HEAD_THREADS) {
        int k = i / HID, u = i % HID;
        float s = 0.f;
        for (int c = 0; c < CELLS_PER_GRID; c++)
            s = fmaf(sdl[c][k], sh[c][u], s);
        gp[i] = s;
    }
    if (tid < NCLS) {
        float s = 0.f;
        for (int c = 0; c < CELLS_PER_GRID; c++)
            s += sdl[c][tid];
        gp[NCLS * HID + tid] = s;
    }
}

// ------------------------------------------------- head of the pair query
//
// The Digit x Size query: two heads on the same hidden layer (fc2 -> 10
// digit classes, fc2s -> 2 size classes), one softmax each, and the soft
// COUNT of every (digit, size) pair, cnt[a][b] = sum_c Pd[c][a] Ps[c][b]
// (Sec. 4 soft group-by over two PE attributes: products of the two
// attributes' probabilities, summed).  With targets: the MSE of the 20
// counts, its backward through both softmaxes down to dh1 (the two heads'
// contributions added before the ReLU mask) and both heads' gradients as
// per-grid partials.
constexpr int NSZ = 2;
constexpr int NH2 = NCLS + NSZ;         // logits of both heads per cell
constexpr int NPRED2 = NCLS * NSZ;      // pair counts per grid
constexpr int H2_PER = NCLS * HID + NCLS + NSZ * HID + NSZ + 1; // partial row

__global__ void __launch_bounds__(HEAD_THREADS) head2_kernel(const bf16 *__restrict__ h1, const float *__restrict__ wd,
                                                             const float *__restrict__ bd,
                                                             const float *__restrict__ ws_,
                                                             const float *__restrict__ bs,
                                                             const float *__restrict__ target, float inv_nout,
                                                             float *__restrict__ logits_d, float *__restrict__ logits_s,
                                                             float *__restrict__ Pd_out, float *__restrict__ Ps_out,
                                                             float *__restrict__ pred_out, bf16 *__restrict__ dh1,
                                                             float *__restrict__ part)
{
    __shared__ float sh[CELLS_PER_GRID][HID];
    __shared__ float sw[NH2][HID];
    __shared__ float sP[CELLS_PER_GRID][NH2]; // logits, then the two softmaxes
    __shared__ float sdl[CELLS_PER_GRID][NH2];
    __shared__ float sdpred[NPRED2];
    const long long grid = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < CELLS_PER_GRID * HID; i += HEAD_THREADS)
        sh[i / HID][i % HID] = bf2f(h1[grid * CELLS_PER_GRID * HID + i]);
    for (int i = tid; i < NH2 * HID; i += HEAD_THREADS)
        sw[i / HID][i % HID] = i < NCLS * HID ? wd[i] : ws_[i - NCLS * HID];
    __syncthreads();
    if (tid < CELLS_PER_GRID * NH2) {
        const int c = tid / NH2, k = tid % NH2;
        float s = k < NCLS ? bd[k] : bs[k - NCLS];
        for (int u = 0; u < HID; u++)
            s = fmaf(sh[c][u], sw[k][u], s);
        sP[c][k] = s;
        const long long cell = grid * CELLS_PER_GRID + c;
        if (k < NCLS && logits_d)
            logits_d[cell * NCLS + k] = s;
        if (k >= NCLS && logits_s)
            logits_s[cell * NSZ + (k - NCLS)] = s;
    }
    __syncthreads();
    if (tid < 2 * CELLS_PER_GRID) { // thread c: digit softmax of cell c; 16 + c: size softmax
        const int c = tid % CELLS_PER_GRID;
        const int k0 = tid < CELLS_PER_GRID ? 0 : NCLS, kn = tid < CELLS_PER_GRID ? NCLS : NSZ;
        float mx = sP[c][k0];
        for (int k = 1; k < kn; k++)
            mx = fmaxf(mx, sP[c][k0 + k]);
        float e[NCLS], z = 0.f;
        for (int k = 0; k < kn; k++) {
            e[k] = expf(sP[c][k0 + k] - mx);
            z += e[k];
        }
        const float iz = 1.0f / z;
        for (int k = 0; k < kn; k++)
            sP[c][k0 + k] = e[k] * iz;
    }
    __syncthreads();
    if (tid < CELLS_PER_GRID * NH2) {
        const int c = tid / NH2, k = tid % NH2;
        const long long cell = grid * CELLS_PER_GRID + c;
        if (k < NCLS && Pd_out)
            Pd_out[cell * NCLS + k] = sP[c][k];
        if (k >= NCLS && Ps_out)
            Ps_out[cell * NSZ + (k - NCLS)] = sP[c][k];
    }
    float d = 0.f;
    if (tid < NPRED2) {
        const int a = tid / NSZ, b = tid % NSZ;
        float s = 0.f;
        for (int c = 0; c < CELLS_PER_GRID; c++)
            s = fmaf(sP[c][a], sP[c][NCLS + b], s);
        if (pred_out)
            pred_out[grid * NPRED2 + tid] = s;
        if (target) {
            d = s - target[grid * NPRED2 + tid];
            sdpred[tid] = 2.f * d * inv_nout;
        }
    }
    if (!target)
        return;
    float *gp = part + grid * H2_PER;
    if (tid < 32) { // the grid's share of the mean loss (lanes >= 20 add 0)
        float l = d * d;
        for (int o = 16; o > 0; o >>= 1)
            l += __shfl_xor_sync(0xffffffffu, l, o);
        if (tid == 0)
            gp[H2_PER - 1] = l * inv_nout;
    }
    __syncthreads();
    if (tid < 2 * CELLS_PER_GRID) {
        const int c = tid % CELLS_PER_GRID;
        if (tid < CELLS_PER_GRID) { // dPd[a] = sum_b dpred[a][b] Ps[c][b], then the softmax backward
            float dP[NCLS], dot = 0.f;
            for (int a = 0; a < NCLS; a++) {
                float v = 0.f;
                for (int b = 0; b < NSZ; b++)
                    v = fmaf(sdpred[a * NSZ + b], sP[c][NCLS + b], v);
                dP[a] = v;
                dot = fmaf(sP[c][a], v, dot);
            }
            for (int a = 0; a < NCLS; a++)
                sdl[c][a] = sP[c][a] * (dP[a] - dot);
        } else { // dPs[b] = sum_a dpred[a][b] Pd[c][a]
            float dP[NSZ], dot = 0.f;
            for (int b = 0; b < NSZ; b++) {
                float v = 0.f;
                for (int a = 0; a < NCLS; a++)
                    v = fmaf(sdpred[a * NSZ + b], sP[c][a], v);
                dP[b] = v;
                dot = fmaf(sP[c][NCLS + b], v, dot);
            }
            for (int b = 0; b < NSZ; b++)
                sdl[c][NCLS + b] = sP[c][NCLS + b] * (dP[b] - dot);
        }
    }
    __syncthreads();
    // dh1[c][u] = (sum_k dl[c][k] w[k][u] over both heads) * (h1 > 0)
    for (int i = tid; i < CELLS_PER_GRID * HID; i += HEAD_THREADS) {
        const int c = i / HID, u = i % HID;
        float s = 0.f;
        for (int k = 0; k < NH2; k++)
            s = fmaf(sdl[c][k], sw[k][u], s);
        dh1[grid * CELLS_PER_GRID * HID + i] = __float2bfloat16_rn(sh[c][u] > 0.f ? s : 0.f);
    }
    // both heads' weight gradients of this grid: [dwd 10x128][dbd 10][dws 2x128][dbs 2][loss]
    for (int i = tid; i < NH2 * HID; i += HEAD_THREADS) {
        const int k = i / HID, u = i % HID;
        float s = 0.f;
        for (int c = 0; c < CELLS_PER_GRID; c++)
            s = fmaf(sdl[c][k], sh[c][u], s);
        gp[k < NCLS ? i : NCLS * HID + NCLS + (i - NCLS * HID)] = s;
    }
    if (tid < NH2) {
        float s = 0.f;
        for (int c = 0; c < CELLS_PER_GRID; c++)
            s += sdl[c][tid];
        gp[tid < NCLS ? NCLS * HID + tid : NCLS * HID + NCLS + NSZ * HID + (tid - NCLS)] = s;
    }
}

// ------------------------------------------------------- exact inference

// Exact query (Sec. 4: the exact operators replace the soft ones at
// inference): argmax of the logits per cell (first maximum), then the exact
// integer COUNT per class and the per-row SUM of class values per grid.
__global__ void exact_count_kernel(const float *__restrict__ logits, long long ngrid, int K, int gh, int gw,
                                   int32_t *__restrict__ labels, long long *__restrict__ cnt,
                                   long long *__restrict__ rsum)
{
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngrid)
        return;
    const int cpg = gh * gw;
    for (int k = 0; k < K; k++)
        cnt[g * K + k] = 0;
    for (int r = 0; r < gh; r++)
        rsum[g * gh + r] = 0;
    for (int c = 0; c < cpg; c++) {
        const float *l = logits + (g * cpg + c) * K;
        int best = 0;
        for (int k = 1; k < K; k++)
            if (l[k] > l[best])
                best = k;
        if (labels)
            labels[g * cpg + c] = best;
        cnt[g * K + best] += 1;
        rsum[g * gh + c / gw] += best;
    }
}

// PE soft group-by (standalone): cnt[g][k] = sum_c P, rsum[g][r] = sum_{c in r} sum_k k P
__global__ void pe_groupby_fwd_kernel(const float *__restrict__ P, long long ngrid, int K, int gh, int gw,
                                      float *__restrict__ cnt, float *__restrict__ rsum)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int cpg = gh * gw;
    if (i >= ngrid * (K + gh))
        return;
    long long g = i / (K + gh);
    int j = (int)(i % (K + gh));
    float s = 0.f;
    if (j < K) {
        for (int c = 0; c < cpg; c++)
            s += P[(g * cpg + c) * K + j];
        cnt[g * K + j] = s;
    } else {
        int r = j - K;
        for (int c = r * gw; c < r * gw + gw; c++)
            for (int k = 0; k < K; k++)
                s = fmaf((float)k, P[(g * cpg + c) * K + k], s);
        rsum[g * gh + r] = s;
    }
}

__global__ void pe_groupby_bwd_kernel(const float *__restrict__ dcnt, const float *__restrict__ drsum, long long ngrid,
                                      int K, int gh, int gw, float *__restrict__ dP)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int cpg = gh * gw;
    if (i >= ngrid * cpg * K)
        return;
    long long cell = i / K;
    int k = (int)(i % K);
    long long g = cell / cpg;
    int r = (int)(cell % cpg) / gw;
    dP[i] = dcnt[g * K + k] + (float)k * drsum[g * gh + r];
}

// Exact pair query: per cell the first arg-max of each attribute's logits,
// then the integer COUNT of every (a, b) pair per grid.
__global__ void exact_count2_kernel(const float *__restrict__ la, int Ka, const float *__restrict__ lb, int Kb,
                                    long long ngrid, int cpg, int32_t *__restrict__ labels_a,
                                    int32_t *__restrict__ labels_b, long long *__restrict__ cnt)
{
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngrid)
        return;
    long long *out = cnt + g * Ka * Kb;
    for (int j = 0; j < Ka * Kb; j++)
        out[j] = 0;
    for (int c = 0; c < cpg; c++) {
        const long long cell = g * cpg + c;
        const float *xa = la + cell * Ka, *xb = lb + cell * Kb;
        int ba = 0, bb = 0;
        for (int k = 1; k < Ka; k++)
            if (xa[k] > xa[ba])
                ba = k;
        for (int k = 1; k < Kb; k++)
            if (xb[k] > xb[bb])
                bb = k;
        if (labels_a)
            labels_a[cell] = ba;
        if (labels_b)
            labels_b[cell] = bb;
        out[ba * Kb + bb] += 1;
    }
}

// Soft pair COUNT: cnt[g][a][b] = sum over the grid's cells of Pa[c][a] Pb[c][b]
__global__ void pe_groupby2_fwd_kernel(const float *__restrict__ Pa, int Ka, const float *__restrict__ Pb, int Kb,
                                       long long ngrid, int cpg, float *__restrict__ cnt)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ngrid * Ka * Kb)
        return;
    const long long g = i / (Ka * Kb);
    const int j = (int)(i % (Ka * Kb)), a = j / Kb, b = j % Kb;
    float s = 0.f;
    for (int c = 0; c < cpg; c++)
        s = fmaf(Pa[(g * cpg + c) * Ka + a], Pb[(g * cpg + c) * Kb + b], s);
    cnt[i] = s;
}

// Its adjoint: dPa[c][a] = sum_b dcnt[g][a][b] Pb[c][b] and
// dPb[c][b] = sum_a dcnt[g][a][b] Pa[c][a]; one thread per element of either.
__global__ void pe_groupby2_bwd_kernel(const float *__restrict__ dcnt, const float *__restrict__ Pa, int Ka,
                                       const float *__restrict__ Pb, int Kb, long long ngrid, int cpg,
                                       float *__restrict__ dPa, float *__restrict__ dPb)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int per = Ka + Kb;
    if (i >= ngrid * cpg * per)
        return;
    const long long cell = i / per;
    const int j = (int)(i % per);
    const float *dc = dcnt + (cell / cpg) * Ka * Kb;
    float s = 0.f;
    if (j < Ka) {
        for (int b = 0; b < Kb; b++)
            s = fmaf(dc[j * Kb + b], Pb[cell * Kb + b], s);
        dPa[cell * Ka + j] = s;
    } else {
        const int b = j - Ka;
        for (int a = 0; a < Ka; a++)
            s = fmaf(dc[a * Kb + b], Pa[cell * Ka + a], s);
        dPb[cell * Kb + b] = s;
    }
}

// ------------------------------------------------------------------- Adam

constexpr int ADAM_MAX = 16;

struct AdamSet {
    float *p[ADAM_MAX];
    const float *g[ADAM_MAX];
    float *m[ADAM_MAX];
    float *v[ADAM_MAX];
    bf16 *copy[ADAM_MAX];
    long long off[ADAM_MAX + 1];
    int count;
};

__global__ void adam_kernel(AdamSet as, float lr, float b1, float b2, float eps, float c1, float c2)
{
    long long total = as.off[as.count];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int t = 0;
        while (i >= as.off[t + 1])
            t++;
        long long j = i - as.off[t];
        float g = as.g[t][j];
        float m = b1 * as.m[t][j] + (1.f - b1) * g;
        float v = b2 * as.v[t][j] + (1.f - b2) * g * g;
        as.m[t][j] = m;
        as.v[t][j] = v;
        float mh = m * c1, vh = v * c2;
        float p = as.p[t][j] - lr * mh / (sqrtf(vh) + eps);
        as.p[t][j] = p;
        if (as.copy[t])
            as.copy[t][j] = __float2bfloat16_rn(p);
    }
}

__global__ void f32_to_bf16_kernel(const float *__restrict__ x, long long n, bf16 *__restrict__ y)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        y[i] = __float2bfloat16_rn(x[i]);
}

} // namespace cnn
} // namespace tdp

using namespace tdp;
using namespace tdp::cnn;

static tdp_status cerr(cudaError_t e) { return e == cudaSuccess ? TDP_OK : TDP_ERR_CUDA; }

static unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// split-K factors (host side) for the fc1 GEMMs and the conv2 weight gradient
static const int FC1_FWD_SPLITS = 9;
static const int FC1_WGRAD_SPLITS = 8;

// CTAs of the conv2 weight gradient: one per SM (each holds 512 tensor-memory
// columns), each writing one partial of dW
static int conv2_wgrad_ctas() { return num_sms(); }

// Resident CTAs per SM of a persistent tcgen05 kernel: as many as the SM's
// shared memory holds (dynamic bytes + its static part and the per-block
// reservation, counted as 2 KiB) and its tensor memory (512 columns) allows.
static int umma_ctas_per_sm(size_t smem, uint32_t tmem_cols)
{
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int by_smem = (int)((size_t)smem_sm / (smem + 2048));
    const int by_tmem = (int)(512 / tmem_cols);
    return std::max(1, std::min(by_smem, by_tmem));
}

extern "C" {

tdp_status tdp_cnn_conv1_fwd(const uint8_t *grids, int64_t n_grids, const float *w1, const float *b1, void *y1,
                             tdp_stream_t stream)
{
    if (n_grids < 0 || (n_grids > 0 && (!grids || !w1 || !b1 || !y1)))
        return TDP_ERR_INVALID_ARG;
    const long long npairs = n_grids * CELLS_PER_GRID * PAIRS_PER_CELL;
    if (npairs == 0)
        return TDP_OK;
    if ((uintptr_t)y1 % 16)
        return TDP_ERR_INVALID_ARG;
    conv1_fwd_kernel<<<blocks_for(npairs, C1F_THREADS), C1F_THREADS, 0, (cudaStream_t)stream>>>(grids, npairs, w1, b1,
                                                                                             (bf16 *)y1);
    return launch_status();
}

tdp_status tdp_cnn_conv2_pool_fwd(const void *y1, int64_t n_cells, const void *w2, const float *b2, void *y2,
                                  uint8_t *argmax, int32_t *d_status, tdp_stream_t stream)
{
    if (n_cells < 0 || (n_cells > 0 && (!y1 || !w2 || !b2 || !y2 || !argmax)))
        return TDP_ERR_INVALID_ARG;
    if (n_cells == 0)
        return TDP_OK;
    // 16-byte alignment of every operand and output row (vector stores, cp.async)
    if (((uintptr_t)y1 | (uintptr_t)w2 | (uintptr_t)y2 | (uintptr_t)argmax) % 16)
        return TDP_ERR_INVALID_ARG;
    const long long ntiles = n_cells * C2_TILES_PER_CELL;
    const size_t smem = (size_t)C2_W_BYTES + C2_WORKERS * C2_STAGE_BYTES;
    if (cudaFuncSetAttribute(conv2_pool_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(conv2_pool_umma_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return TDP_ERR_CUDA;
    const long long grid = std::min<long long>(ntiles, (long long)umma_ctas_per_sm(smem, C2_TMEM_ALLOC) * num_sms());
    conv2_pool_umma_kernel<<<(unsigned)grid, C2_THREADS, smem, (cudaStream_t)stream>>>(
        (const bf16 *)y1, (const bf16 *)w2, b2, (bf16 *)y2, argmax, ntiles, d_status, spin_limit());
    return launch_status();
}

size_t tdp_cnn_fc1_fwd_workspace(int64_t n_cells)
{
    return align_up((size_t)FC1_FWD_SPLITS * n_cells * HID * sizeof(float), 256);
}

tdp_status tdp_cnn_fc1_fwd(const void *y2, int64_t n_cells, const void *wfc1, const float *bfc1, void *h1, void *ws,
                           size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n_cells < 0 || (n_cells > 0 && (!y2 || !wfc1 || !bfc1 || !h1)))
        return TDP_ERR_INVALID_ARG;
    if (((uintptr_t)y2 | (uintptr_t)wfc1) % 16)
        return TDP_ERR_INVALID_ARG;
    if (n_cells == 0)
        return TDP_OK;
    if (!ws || ws_bytes < tdp_cnn_fc1_fwd_workspace(n_cells))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    float *part = (float *)ws;
    const int M = (int)n_cells;
    const GemmOp la{y2, M, FEAT, FEAT, false}, lb{wfc1, HID, FEAT, FEAT, false};
    EpiPartialF32 epi{part, M, HID, (size_t)M * HID};
    tdp_status st = launch_umma_gemm<HID, 3, false, false>(la, lb, epi, M, HID, FEAT, FC1_FWD_SPLITS, d_status, s);
    if (st != TDP_OK)
        return st;
    long long n = (long long)M * HID;
    splitk_reduce_kernel<<<blocks_for(n, 256), 256, 0, s>>>(part, FC1_FWD_SPLITS, (size_t)M * HID, n, HID, bfc1, 1,
                                                            (bf16 *)h1, nullptr);
    return launch_status();
}

size_t tdp_cnn_head_workspace(int64_t n_grids)
{
    return align_up((size_t)n_grids * (NCLS * HID + NCLS + 1) * sizeof(float), 256);
}

tdp_status tdp_cnn_head(const void *h1, int64_t n_grids, const float *wfc2, const float *bfc2, const float *targets,
                        float *logits, float *P, float *pred, void *dh1, float *dwfc2, float *dbfc2, float *loss,
                        void *ws, size_t ws_bytes, tdp_stream_t stream)
{
    if (n_grids < 0 || (n_grids > 0 && (!h1 || !wfc2 || !bfc2)))
        return TDP_ERR_INVALID_ARG;
    if (targets && (!dh1 || !dwfc2 || !dbfc2 || !loss))
        return TDP_ERR_INVALID_ARG;
    if (n_grids == 0)
        return TDP_OK;
    if (targets && (!ws || ws_bytes < tdp_cnn_head_workspace(n_grids)))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    float *part = (float *)ws;
    head_kernel<<<(unsigned)n_grids, HEAD_THREADS, 0, s>>>((const bf16 *)h1, n_grids, wfc2, bfc2, targets,
                                                           1.0f / (float)(n_grids * NPRED), logits, P, pred,
                                                           (bf16 *)dh1, part);
    if (targets) {
        const size_t per = NCLS * HID + NCLS + 1;
        // one launch: fc2 weight sums, then the 10 bias sums, then the loss
        partial_sum_kernel<<<psum_blocks((int)per), 32 * PS_SLICES, 0, s>>>(
            part, (int)n_grids, (int)per, per, PsOut{dwfc2, dbfc2, loss, NCLS * HID, NCLS});
    }
    return launch_status();
}

size_t tdp_cnn_head2_workspace(int64_t n_grids)
{
    return align_up((size_t)n_grids * H2_PER * sizeof(float), 256);
}

tdp_status tdp_cnn_head2(const void *h1, int64_t n_grids, const float *wfc2, const float *bfc2, const float *wfc2s,
                         const float *bfc2s, const float *targets, float *logits, float *logits_s, float *P,
                         float *Ps, float *pred, void *dh1, float *dwfc2, float *dbfc2, float *dwfc2s,
                         float *dbfc2s, float *loss, void *ws, size_t ws_bytes, tdp_stream_t stream)
{
    if (n_grids < 0 || (n_grids > 0 && (!h1 || !wfc2 || !bfc2 || !wfc2s || !bfc2s)))
        return TDP_ERR_INVALID_ARG;
    if (targets && (!dh1 || !dwfc2 || !dbfc2 || !dwfc2s || !dbfc2s || !loss))
        return TDP_ERR_INVALID_ARG;
    if (n_grids == 0)
        return TDP_OK;
    if (targets && (!ws || ws_bytes < tdp_cnn_head2_workspace(n_grids)))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    float *part = (float *)ws;
    head2_kernel<<<(unsigned)n_grids, HEAD_THREADS, 0, s>>>((const bf16 *)h1, wfc2, bfc2, wfc2s, bfc2s, targets,
                                                            1.0f / (float)(n_grids * NPRED2), logits, logits_s, P,
                                                            Ps, pred, (bf16 *)dh1, part);
    if (targets) {
        // digit head's weight and bias sums, then the size head's and the loss
        const int n1 = NCLS * HID + NCLS, n2 = NSZ * HID + NSZ + 1;
        partial_sum_kernel<<<psum_blocks(n1), 32 * PS_SLICES, 0, s>>>(part, (int)n_grids, n1, H2_PER,
                                                                      PsOut{dwfc2, dbfc2, nullptr, NCLS * HID, NCLS});
        partial_sum_kernel<<<psum_blocks(n2), 32 * PS_SLICES, 0, s>>>(part + n1, (int)n_grids, n2, H2_PER,
                                                                      PsOut{dwfc2s, dbfc2s, loss, NSZ * HID, NSZ});
    }
    return launch_status();
}

size_t tdp_cnn_fc1_bwd_workspace(int64_t n_cells)
{
    size_t a = align_up((size_t)FC1_WGRAD_SPLITS * HID * FEAT * sizeof(float), 256);
    size_t b = align_up((size_t)colsum_blocks(n_cells, HID) * HID * sizeof(float), 256);
    return a + b;
}

tdp_status tdp_cnn_fc1_bwd(const void *dh1, const void *y2, const void *wfc1, int64_t n_cells, void *dy2p,
                           float *dwfc1, float *dbfc1, void *ws, size_t ws_bytes, int32_t *d_status,
                           tdp_stream_t stream)
{
    if (n_cells < 1 || !dh1 || !y2 || !wfc1 || !dy2p || !dwfc1 || !dbfc1)
        return TDP_ERR_INVALID_ARG;
    if (((uintptr_t)dh1 | (uintptr_t)y2 | (uintptr_t)wfc1 | (uintptr_t)dy2p) % 16)
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_cnn_fc1_bwd_workspace(n_cells))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const int M = (int)n_cells;
    // dgrad: dy2p[cell][f] = (sum_u dh1[cell][u] wfc1[u][f]) * (y2 > 0)
    {
        const GemmOp la{dh1, M, HID, HID, false}, lb{wfc1, FEAT, HID, FEAT, true};
        EpiMaskedBf16 epi{(bf16 *)dy2p, (const bf16 *)y2, M, FEAT, EpiMaskedBf16::pitch(128)};
        tdp_status st = launch_umma_gemm<128, 2, false, true>(la, lb, epi, M, FEAT, HID, 1, d_status, s);
        if (st != TDP_OK)
            return st;
    }
    // wgrad: dwfc1[u][f] = sum_cell dh1[cell][u] y2[cell][f]
    float *part = (float *)ws;
    {
        const GemmOp la{dh1, HID, M, HID, true}, lb{y2, FEAT, M, FEAT, true};
        EpiPartialF32 epi{part, HID, FEAT, (size_t)HID * FEAT};
        tdp_status st = launch_umma_gemm<256, 2, true, true>(la, lb, epi, HID, FEAT, M, FC1_WGRAD_SPLITS, d_status, s);
        if (st != TDP_OK)
            return st;
        long long n = (long long)HID * FEAT;
        splitk_reduce_kernel<<<blocks_for(n, 256), 256, 0, s>>>(part, FC1_WGRAD_SPLITS, (size_t)HID * FEAT, n, FEAT,
                                                                nullptr, 0, nullptr, dwfc1);
    }
    // bias: column sums of dh1
    {
        float *bp = (float *)((char *)ws + align_up((size_t)FC1_WGRAD_SPLITS * HID * FEAT * sizeof(float), 256));
        const int nb = colsum_blocks(n_cells, HID);
        colsum_bf16_kernel<<<nb, CS_THREADS, 0, s>>>((const bf16 *)dh1, n_cells, HID, bp);
        partial_sum_kernel<<<psum_blocks(HID), 32 * PS_SLICES, 0, s>>>(bp, nb, HID, HID, ps_out(dbfc1));
    }
    return launch_status();
}

size_t tdp_cnn_conv2_bwd_workspace(int64_t n_cells)
{
    int sp = conv2_wgrad_ctas();
    long long Q = n_cells * PO * PO;
    size_t a = align_up((size_t)sp * CH2 * 9 * CH1 * sizeof(float), 256);
    size_t b = align_up((size_t)colsum_blocks(Q, CH2) * CH2 * sizeof(float), 256);
    return a + b;
}

tdp_status tdp_cnn_conv2_bwd(const void *dy2p, const uint8_t *argmax, const void *y1, const void *w2, int64_t n_cells,
                             void *dz1, float *dw2, float *db2, void *ws, size_t ws_bytes, int32_t *d_status,
                             tdp_stream_t stream)
{
    if (n_cells < 1 || !dy2p || !argmax || !y1 || !w2 || !dw2 || !db2)
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_cnn_conv2_bwd_workspace(n_cells))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    // 16-byte alignment of the activation rows (vector loads and stores)
    if (((uintptr_t)dy2p | (uintptr_t)argmax | (uintptr_t)y1 | (uintptr_t)dz1) % 16)
        return TDP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // dgrad (optional): dz1[cell][y][x][ci] = (sum dz2 * w2) * (y1 > 0), tcgen05
    if (dz1) {
        const long long ntiles = n_cells * DG_TILES_PER_CELL;
        const size_t smem = (size_t)DG_W_BYTES + DG_WORKERS * DG_PATCH_BYTES;
        if (cudaFuncSetAttribute(conv2_dgrad_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(conv2_dgrad_umma_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return TDP_ERR_CUDA;
        const long long grid =
            std::min<long long>(ntiles, (long long)umma_ctas_per_sm(smem, DG_TMEM_ALLOC) * num_sms());
        conv2_dgrad_umma_kernel<<<(unsigned)grid, DG_THREADS, smem, s>>>(
            (const bf16 *)dy2p, argmax, (const bf16 *)w2, (const bf16 *)y1, (bf16 *)dz1, ntiles, d_status,
            spin_limit());
        if (cudaGetLastError() != cudaSuccess)
            return TDP_ERR_CUDA;
    }
    // wgrad: dw2[co][(ky,kx,ci)] = sum_p dz2[p][co] y1[p+(ky,kx)][ci], tcgen05, one
    // fp32 partial per CTA summed in block order
    const int sp = conv2_wgrad_ctas();
    float *part = (float *)ws;
    {
        const long long ntiles = n_cells * WG_TILES_PER_CELL;
        const size_t smem = (size_t)WG_PRODUCERS * WG_BUF_BYTES;
        if (cudaFuncSetAttribute(conv2_wgrad_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(conv2_wgrad_umma_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return TDP_ERR_CUDA;
        const int grid = (int)std::min<long long>(ntiles, sp);
        conv2_wgrad_umma_kernel<<<grid, WG_THREADS, smem, s>>>((const bf16 *)dy2p, argmax, (const bf16 *)y1, ntiles,
                                                               part, d_status, spin_limit());
        partial_sum_kernel<<<psum_blocks(CH2 * 9 * CH1), 32 * PS_SLICES, 0, s>>>(part, grid, CH2 * 9 * CH1,
                                                                                 CH2 * 9 * CH1, ps_out(dw2));
    }
    // bias: sum of the pooled gradient (each pooled value lands on exactly one pixel)
    {
        float *bp = (float *)((char *)ws + align_up((size_t)sp * CH2 * 9 * CH1 * sizeof(float), 256));
        long long Q = n_cells * PO * PO;
        const int nb = colsum_blocks(Q, CH2);
        colsum_bf16_kernel<<<nb, CS_THREADS, 0, s>>>((const bf16 *)dy2p, Q, CH2, bp);
        partial_sum_kernel<<<psum_blocks(CH2), 32 * PS_SLICES, 0, s>>>(bp, nb, CH2, CH2, ps_out(db2));
    }
    return launch_status();
}

size_t tdp_cnn_conv1_bwd_workspace(int64_t n_cells)
{
    (void)n_cells;
    return align_up((size_t)W1_BLOCKS_PER_SM * num_sms() * CH1 * 10 * sizeof(float), 256);
}

tdp_status tdp_cnn_conv1_bwd(const void *dz1, const uint8_t *grids, int64_t n_cells, float *dw1, float *db1, void *ws,
                             size_t ws_bytes, tdp_stream_t stream)
{
    if (n_cells < 1 || n_cells % CELLS_PER_GRID || !dz1 || !grids || !dw1 || !db1)
        return TDP_ERR_INVALID_ARG;
    if (!ws || ws_bytes < tdp_cnn_conv1_bwd_workspace(n_cells))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if ((uintptr_t)dz1 % 4)
        return TDP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // cells spread evenly over the resident blocks
    const long long cap = (long long)W1_BLOCKS_PER_SM * num_sms();
    const long long cpb = (n_cells + cap - 1) / cap;
    const int nb = (int)((n_cells + cpb - 1) / cpb);
    float *part = (float *)ws;
    conv1_wgrad_kernel<<<nb, W1_THREADS, 0, s>>>((const bf16 *)dz1, grids, n_cells, cpb, part);
    // each partial row: 288 weight sums, then the 32 bias sums
    // one launch: the 288 weight sums, then the 32 bias sums
    partial_sum_kernel<<<psum_blocks(CH1 * 10), 32 * PS_SLICES, 0, s>>>(part, nb, CH1 * 10, CH1 * 10,
                                                                        PsOut{dw1, db1, nullptr, CH1 * 9, CH1});
    return launch_status();
}

tdp_status tdp_adam_step(float *const *params, const float *const *grads, float *const *m, float *const *v,
                         void *const *bf16_copies, const int64_t *sizes, int32_t count, int32_t step, float lr,
                         float beta1, float beta2, float eps, tdp_stream_t stream)
{
    if (count < 1 || count > ADAM_MAX || step < 1 || !params || !grads || !m || !v || !sizes)
        return TDP_ERR_INVALID_ARG;
    AdamSet as;
    as.count = count;
    as.off[0] = 0;
    for (int i = 0; i < ADAM_MAX; i++) {
        bool on = i < count;
        as.p[i] = on ? params[i] : nullptr;
        as.g[i] = on ? grads[i] : nullptr;
        as.m[i] = on ? m[i] : nullptr;
        as.v[i] = on ? v[i] : nullptr;
        as.copy[i] = on && bf16_copies ? (bf16 *)bf16_copies[i] : nullptr;
        if (on && (!as.p[i] || !as.g[i] || !as.m[i] || !as.v[i] || sizes[i] < 0))
            return TDP_ERR_INVALID_ARG;
        as.off[i + 1] = as.off[i] + (on ? sizes[i] : 0);
    }
    long long total = as.off[count];
    if (total == 0)
        return TDP_OK;
    float c1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
    float c2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
    unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, (long long)num_sms() * 8);
    adam_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(as, lr, beta1, beta2, eps, c1, c2);
    return launch_status();
}

tdp_status tdp_f32_to_bf16(const float *x, int64_t n, void *y, tdp_stream_t stream)
{
    if (n < 0 || (n > 0 && (!x || !y)))
        return TDP_ERR_INVALID_ARG;
    if (n == 0)
        return TDP_OK;
    f32_to_bf16_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(x, n, (bf16 *)y);
    return launch_status();
}

tdp_status tdp_exact_pe_count(const float *logits, int64_t n_grids, int32_t K, int32_t grid_h, int32_t grid_w,
                              int32_t *labels, int64_t *cnt, int64_t *rsum, tdp_stream_t stream)
{
    if (n_grids < 0 || K < 1 || grid_h < 1 || grid_w < 1 || (n_grids > 0 && (!logits || !cnt || !rsum)))
        return TDP_ERR_INVALID_ARG;
    if (n_grids == 0)
        return TDP_OK;
    exact_count_kernel<<<blocks_for(n_grids, 128), 128, 0, (cudaStream_t)stream>>>(
        logits, n_grids, K, grid_h, grid_w, labels, (long long *)cnt, (long long *)rsum);
    return launch_status();
}

tdp_status tdp_pe_groupby_fwd(const float *P, int64_t n_grids, int32_t K, int32_t grid_h, int32_t grid_w, float *cnt,
                              float *rsum, tdp_stream_t stream)
{
    if (n_grids < 0 || K < 1 || grid_h < 1 || grid_w < 1 || (n_grids > 0 && (!P || !cnt || !rsum)))
        return TDP_ERR_INVALID_ARG;
    long long n = n_grids * (K + grid_h);
    if (n == 0)
        return TDP_OK;
    pe_groupby_fwd_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(P, n_grids, K, grid_h, grid_w, cnt,
                                                                                rsum);
    return launch_status();
}

tdp_status tdp_pe_groupby_bwd(const float *dcnt, const float *drsum, int64_t n_grids, int32_t K, int32_t grid_h,
                              int32_t grid_w, float *dP, tdp_stream_t stream)
{
    if (n_grids < 0 || K < 1 || grid_h < 1 || grid_w < 1 || (n_grids > 0 && (!dcnt || !drsum || !dP)))
        return TDP_ERR_INVALID_ARG;
    long long n = n_grids * grid_h * grid_w * K;
    if (n == 0)
        return TDP_OK;
    pe_groupby_bwd_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(dcnt, drsum, n_grids, K, grid_h,
                                                                                grid_w, dP);
    return launch_status();
}

tdp_status tdp_exact_pe_count2(const float *logits_a, int32_t Ka, const float *logits_b, int32_t Kb, int64_t n_grids,
                               int32_t cells, int32_t *labels_a, int32_t *labels_b, int64_t *cnt,
                               tdp_stream_t stream)
{
    if (n_grids < 0 || Ka < 1 || Kb < 1 || cells < 1 || (n_grids > 0 && (!logits_a || !logits_b || !cnt)))
        return TDP_ERR_INVALID_ARG;
    if (n_grids == 0)
        return TDP_OK;
    exact_count2_kernel<<<blocks_for(n_grids, 128), 128, 0, (cudaStream_t)stream>>>(
        logits_a, Ka, logits_b, Kb, n_grids, cells, labels_a, labels_b, (long long *)cnt);
    return launch_status();
}

tdp_status tdp_pe_groupby2_fwd(const float *Pa, int32_t Ka, const float *Pb, int32_t Kb, int64_t n_grids,
                               int32_t cells, float *cnt, tdp_stream_t stream)
{
    if (n_grids < 0 || Ka < 1 || Kb < 1 || cells < 1 || (n_grids > 0 && (!Pa || !Pb || !cnt)))
        return TDP_ERR_INVALID_ARG;
    const long long n = n_grids * Ka * Kb;
    if (n == 0)
        return TDP_OK;
    pe_groupby2_fwd_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(Pa, Ka, Pb, Kb, n_grids, cells,
                                                                                 cnt);
    return launch_status();
}

tdp_status tdp_pe_groupby2_bwd(const float *dcnt, const float *Pa, int32_t Ka, const float *Pb, int32_t Kb,
                               int64_t n_grids, int32_t cells, float *dPa, float *dPb, tdp_stream_t stream)
{
    if (n_grids < 0 || Ka < 1 || Kb < 1 || cells < 1 ||
        (n_grids > 0 && (!dcnt || !Pa || !Pb || !dPa || !dPb)))
        return TDP_ERR_INVALID_ARG;
    const long long n = n_grids * cells * (Ka + Kb);
    if (n == 0)
        return TDP_OK;
    pe_groupby2_bwd_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(dcnt, Pa, Ka, Pb, Kb, n_grids,
                                                                                 cells, dPa, dPb);
    return launch_status();
}

} // extern "C"
