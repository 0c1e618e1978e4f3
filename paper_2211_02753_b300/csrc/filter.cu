// K1/K2: predicate filter with stream compaction and fused column gather.
//
// One cooperative launch of as many blocks as fit on the GPU at once.  Block
// b owns a contiguous chunk of rows; the chunks of all blocks form a round,
// and a table larger than one round (G blocks x FT_MASK_BYTES*8 rows) takes
// several.  Per round:
//   1. count: the chunk streams through a ring of FT_STAGES shared-memory
//      tiles of TILE = 256 x 4 x STEPS rows (one bulk copy per predicate
//      column per tile, cp.async.bulk with completion on the stage's
//      mbarrier, issued FT_STAGES tiles ahead; ragged tiles and columns whose
//      base is not 16-byte aligned are read with plain loads).  Thread t
//      tests the 4 x STEPS consecutive rows t*4*STEPS.. of each tile with
//      range tests (lo <= v <= hi) != neg on the column's own type and keeps
//      the result as one mask bit per row in shared memory.  The block
//      publishes its count.
//   2. one grid-wide barrier (bounded wait).  The block's output offset is
//      the sum of the counts of the chunks before it.
//   3. write: for each tile of the chunk, a popc of each thread's mask word,
//      a warp shuffle scan and the 8 warp totals rank the qualifying rows;
//      their tile-local indices are staged in shared memory and the block
//      writes the run of row ids, and the gathered columns at those rows, to
//      consecutive output slots (coalesced stores).
// The predicate columns are read once and the row ids written once (the
// algorithmic bytes); no tile waits on another tile's prefix, so the only
// cross-block wait is the one barrier per round.  Output is stable.
#include <algorithm>

#include "filter_api.cuh"

namespace tdp {

constexpr int FT_THREADS = 256;
constexpr int FT_STAGES = 2;
constexpr int FT_MAX_STEPS = 8;
constexpr int FT_MASK_BYTES = 18 * 1024;    // mask bits of one chunk: 147456 rows
constexpr int FT_MIN_TILE = FT_THREADS * 4; // 1024 rows
constexpr int FT_WROWS = 4096;              // rows per write batch (a stage holds their ids)

// Clears the mask bits of the thread's rows r0 + 4j + 0..3 (j < STEPS) that
// fail predicate p; the tile of the column is in shared memory.
template <int STEPS>
__device__ __forceinline__ void ft_test_smem(const PredSet &ps, int p, const unsigned char *col, int r0, unsigned &m)
{
    const int dt = ps.dt[p];
    const unsigned neg = (unsigned)ps.neg[p];
    unsigned t = 0;
    if (dt == TDP_I64) {
        const long long lo = ps.lo[p];
        const unsigned long long span = (unsigned long long)(ps.hi[p] - lo);
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            const longlong2 *q = (const longlong2 *)(col + (size_t)(r0 + 4 * j) * 8);
            const longlong2 a = q[0], b = q[1];
            t |= (range_holds64(a.x, lo, span, neg) | range_holds64(a.y, lo, span, neg) << 1 |
                  range_holds64(b.x, lo, span, neg) << 2 | range_holds64(b.y, lo, span, neg) << 3)
                 << (4 * j);
        }
    } else if (dt == TDP_I32) {
        const int lo = (int)ps.lo[p];
        const unsigned span = (unsigned)((int)ps.hi[p] - lo);
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            const int4 w = *(const int4 *)(col + (size_t)(r0 + 4 * j) * 4);
            t |= (range_holds32(w.x, lo, span, neg) | range_holds32(w.y, lo, span, neg) << 1 |
                  range_holds32(w.z, lo, span, neg) << 2 | range_holds32(w.w, lo, span, neg) << 3)
                 << (4 * j);
        }
    } else {
        const int lo = (int)ps.lo[p];
        const unsigned span = (unsigned)((int)ps.hi[p] - lo);
        const bool sgn = dt == TDP_I8;
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            const unsigned w = *(const unsigned *)(col + r0 + 4 * j);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned b = (w >> (8 * k)) & 0xffu;
                const int v = sgn ? (int)(int8_t)b : (int)b;
                t |= range_holds32(v, lo, span, neg) << (4 * j + k);
            }
        }
    }
    m &= t;
}

// Same for rows read from global memory (ragged tile or unaligned column).
template <int STEPS>
__device__ __forceinline__ void ft_test_global(const PredSet &ps, int p, long long r0, long long n, unsigned &m)
{
    const unsigned neg = (unsigned)ps.neg[p];
    const long long lo = ps.lo[p];
    const unsigned long long span = (unsigned long long)(ps.hi[p] - lo);
    unsigned t = 0;
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        long long v[4];
        load4_int(ps.col[p], ps.dt[p], ps.vec_ok[p], r0 + 4 * j, n, v);
#pragma unroll
        for (int k = 0; k < 4; k++)
            t |= range_holds64(v[k], lo, span, neg) << (4 * j + k);
    }
    m &= t;
}

// Whether the tile of rows [base, base + TILE) is staged by bulk copies.
__device__ __forceinline__ bool ft_bulk(const PredSet &ps, long long base, long long tile_rows, long long n)
{
    bool bulk = ps.n > 0 && base + tile_rows <= n;
    for (int p = 0; p < ps.n; p++)
        bulk = bulk && ps.vec_ok[p];
    return bulk;
}

// Stages the tile at row `base` (one bulk copy per predicate column) into a
// ring stage, or only arrives when the tile is read with plain loads.  One
// thread calls it.
template <int STEPS>
__device__ __forceinline__ void ft_stage(const PredSet &ps, unsigned char *stage, uint32_t stage_bytes, uint64_t *bar,
                                         long long base, long long n)
{
    constexpr int TILE = FT_THREADS * 4 * STEPS;
    if (!ft_bulk(ps, base, TILE, n)) {
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    // the stage's previous contents were read by generic loads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the transaction count is exactly the bytes copied (the stage may be larger)
    uint32_t tile_bytes = 0;
    for (int p = 0; p < ps.n; p++)
        tile_bytes += TILE * (uint32_t)dtype_size_dev(ps.dt[p]);
    mbar_arrive_expect_tx(bar, tile_bytes);
    uint32_t off = 0;
    for (int p = 0; p < ps.n; p++) {
        const uint32_t sz = TILE * (uint32_t)dtype_size_dev(ps.dt[p]);
        bulk_load(stage + off, (const char *)ps.col[p] + (size_t)base * dtype_size_dev(ps.dt[p]), sz, bar);
        off += sz;
    }
}

template <int STEPS>
__global__ void __launch_bounds__(FT_THREADS, 4) filter_kernel(PredSet ps, GatherSet gs, long long n_host,
                                                            const long long *d_n, int32_t *out_rowid, long long cap,
                                                            long long *d_count, unsigned long long *counts,
                                                            unsigned *barrier, int32_t *d_status, uint32_t limit,
                                                            uint32_t stage_bytes, long long chunk_rows, int rounds)
{
    constexpr int TILE = FT_THREADS * 4 * STEPS;
    constexpr int RPT = 4 * STEPS; // rows per thread per tile
    extern __shared__ __align__(128) unsigned char ft_smem[];
    __shared__ __align__(8) uint64_t s_bar[FT_STAGES];
    __shared__ unsigned s_warp[FT_THREADS / 32];
    __shared__ unsigned long long s_off[2];

    const long long n = d_n ? min(*d_n, n_host) : n_host;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = threadIdx.x * RPT;
    unsigned *bitmap = (unsigned *)(ft_smem + (size_t)FT_STAGES * stage_bytes); // one bit per chunk row
    // row ids leave by bulk copies from the ring when there is nothing to
    // gather and the output is 16-byte aligned
    const bool bulk_out = out_rowid && gs.n == 0 && ((uintptr_t)out_rowid % 16) == 0;

    if (threadIdx.x == 0)
        for (int s = 0; s < FT_STAGES; s++)
            mbar_init(&s_bar[s], 1);
    __syncthreads();

    bool lost = false;             // a stage wait ran out (its copy may still land)
    unsigned long long before = 0; // rows selected by earlier rounds
    long long use = 0;             // ring uses so far (stage = use % FT_STAGES)
    for (int round = 0; round < rounds; round++) {
        const long long c0 = ((long long)round * G + b) * chunk_rows; // chunk start
        const long long c1 = min(c0 + chunk_rows, n);
        const int nt = c1 > c0 ? (int)((c1 - c0 + TILE - 1) / TILE) : 0;

        // 1. count
        if (threadIdx.x == 0)
            for (int k = 0; k < min(nt, FT_STAGES); k++) {
                const int st = (int)((use + k) % FT_STAGES);
                ft_stage<STEPS>(ps, ft_smem + (size_t)st * stage_bytes, stage_bytes, &s_bar[st], c0 + (long long)k * TILE,
                                n);
            }
        unsigned cnt = 0;
        for (int k = 0; k < nt; k++) {
            const long long u = use + k;
            const int st = (int)(u % FT_STAGES);
            unsigned char *stage = ft_smem + (size_t)st * stage_bytes;
            const long long base = c0 + (long long)k * TILE;
            if (!mbar_wait(&s_bar[st], (uint32_t)(u / FT_STAGES) & 1u, limit)) {
                set_status(d_status, TDP_ERR_TIMEOUT); // results are void; no hang
                lost = true;
            }
            const long long left = n - base - r0;
            unsigned m = left >= RPT ? (RPT == 32 ? 0xffffffffu : (1u << RPT) - 1u)
                                     : (left > 0 ? (1u << left) - 1u : 0u);
            if (ft_bulk(ps, base, TILE, n)) {
                uint32_t off = 0;
                for (int p = 0; p < ps.n; p++) {
                    ft_test_smem<STEPS>(ps, p, stage + off, r0, m);
                    off += TILE * dtype_size_dev(ps.dt[p]);
                }
            } else {
                for (int p = 0; p < ps.n; p++)
                    ft_test_global<STEPS>(ps, p, base + r0, n, m);
            }
            cnt += __popc(m);
            // row-order bitmap: the 32 / RPT lanes of a group OR their bits
            // into one 32-bit word (rows t*RPT.. are consecutive)
            {
                constexpr int GL = 32 / RPT;
                unsigned w = RPT == 32 ? m : m << (RPT * (lane % GL));
#pragma unroll
                for (int o = 1; o < GL; o <<= 1)
                    w |= __shfl_xor_sync(0xffffffffu, w, o);
                if (lane % GL == 0)
                    bitmap[(k * TILE + r0) / 32] = w;
            }
            __syncthreads(); // stage consumed
            if (threadIdx.x == 0 && k + FT_STAGES < nt)
                ft_stage<STEPS>(ps, stage, stage_bytes, &s_bar[st], base + (long long)FT_STAGES * TILE, n);
        }
        use += nt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0)
            s_warp[warp] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < FT_THREADS / 32; w++)
                t += s_warp[w];
            counts[(size_t)round * G + b] = t;
        }

        // 2. one barrier; the chunk's offset
        grid_barrier(barrier, (unsigned)G * (round + 1), limit, d_status);
        if (warp == 0) {
            unsigned long long lo = 0, all = 0;
            for (int i = lane; i < G; i += 32) {
                const unsigned long long v = ld_relaxed_u64(&counts[(size_t)round * G + i]);
                all += v;
                lo += i < b ? v : 0ull;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo += __shfl_xor_sync(0xffffffffu, lo, o);
                all += __shfl_xor_sync(0xffffffffu, all, o);
            }
            if (lane == 0) {
                s_off[0] = before + lo;
                s_off[1] = all;
            }
        }
        __syncthreads();
        unsigned long long excl = s_off[0];
        before += s_off[1];

        // 3. write
        const int nwords = (int)((c1 - c0 + 31) / 32);
        if (bulk_out) {
            // Row ids only, to a 16-byte aligned output: batches of
            // FT_WROWS rows.  Warp w ranks the rows of its FT_WROWS/256
            // bitmap words (lanes = the 32 rows of a word) and stores their
            // ids in a ring stage at their slot's position modulo 4, so that
            // the batch's 16-byte aligned body leaves by one bulk copy; the
            // at most 3 ids before and after it are plain stores.
            constexpr int WPW = FT_WROWS / 32 / (FT_THREADS / 32); // words per warp per batch
            const unsigned lt = lanemask_lt();
            for (int wb = 0, bi = 0; wb < nwords; wb += FT_WROWS / 32, bi++) {
                const int ws0 = wb + warp * WPW;
                unsigned bm[WPW];
                unsigned wc = 0;
#pragma unroll
                for (int j = 0; j < WPW; j++) {
                    bm[j] = ws0 + j < nwords ? bitmap[ws0 + j] : 0u;
                    wc += __popc(bm[j]);
                }
                if (lane == 0)
                    s_warp[warp] = wc;
                if (threadIdx.x == 32)
                    bulk_wait_read<1>(); // the batch two back has left this stage
                __syncthreads();
                unsigned woff = 0, tot = 0;
#pragma unroll
                for (int w = 0; w < FT_THREADS / 32; w++) {
                    const unsigned t = s_warp[w];
                    woff += w < warp ? t : 0;
                    tot += t;
                }
                const long long e = (long long)excl;
                const int pad = (int)(e & 3);
                int32_t *stg = (int32_t *)(ft_smem + (size_t)(bi & 1) * stage_bytes);
                unsigned q = pad + woff;
#pragma unroll
                for (int j = 0; j < WPW; j++) {
                    if (bm[j] >> lane & 1u)
                        stg[q + __popc(bm[j] & lt)] = (int32_t)(c0 + (long long)(ws0 + j) * 32 + lane);
                    q += __popc(bm[j]);
                }
                fence_proxy_async_smem();
                __syncthreads(); // ids staged
                const long long t = max(0ll, min((long long)tot, cap - e));
                const long long head = min(t, (long long)((4 - pad) & 3));
                const long long body = (t - head) & ~3ll;
                if (threadIdx.x < head)
                    out_rowid[e + threadIdx.x] = stg[pad + threadIdx.x];
                else if (threadIdx.x >= 64 && threadIdx.x - 64 < t - head - body)
                    out_rowid[e + head + body + (threadIdx.x - 64)] = stg[pad + head + body + (threadIdx.x - 64)];
                if (threadIdx.x == 32 && body > 0) {
                    bulk_store(out_rowid + e + head, stg + pad + head, (uint32_t)(body * 4));
                    bulk_commit();
                }
                excl += tot;
            }
            if (threadIdx.x == 32)
                bulk_wait_all();
        } else {
            // warp w walks its contiguous share of the chunk's bitmap words
            // in row order; the selected lanes of a 32-row word store at
            // consecutive slots (rank = popc of the lower lanes' bits)
            // shares in whole groups of 4 words (16-byte loads of the bitmap)
            const int per = ((nwords + FT_THREADS / 32 - 1) / (FT_THREADS / 32) + 3) & ~3;
            const int w0 = min(nwords, warp * per), w1 = min(nwords, w0 + per);
            unsigned wc = 0;
            for (int i = w0 + lane; i < w1; i += 32)
                wc += __popc(bitmap[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                wc += __shfl_xor_sync(0xffffffffu, wc, o);
            if (lane == 0)
                s_warp[warp] = wc;
            __syncthreads();
            long long pos = (long long)excl;
            unsigned long long btot = 0;
#pragma unroll
            for (int w = 0; w < FT_THREADS / 32; w++) {
                pos += w < warp ? (long long)s_warp[w] : 0ll;
                btot += s_warp[w];
            }
            const unsigned lt = lanemask_lt();
            for (int i = w0; i < w1; i += 4) {
                // words past w1 are read as 0: the bitmap has whole tiles of
                // words (a multiple of 4) and the share ends on a group of 4
                // or at the chunk's last word
                const uint4 q4 = *(const uint4 *)(bitmap + i);
                unsigned bm[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (i + j >= w1)
                        bm[j] = 0u;
                    const long long q = pos + __popc(bm[j] & lt);
                    const long long row = c0 + (long long)(i + j) * 32 + lane;
                    if ((bm[j] >> lane & 1u) && q < cap) {
                        if (out_rowid)
                            out_rowid[q] = (int32_t)row;
                        for (int g = 0; g < gs.n; g++) {
                            switch (gs.size[g]) {
                            case 8: ((long long *)gs.out[g])[q] = __ldg((const long long *)gs.col[g] + row); break;
                            case 4: ((int32_t *)gs.out[g])[q] = __ldg((const int32_t *)gs.col[g] + row); break;
                            case 2: ((uint16_t *)gs.out[g])[q] = ((const uint16_t *)gs.col[g])[row]; break;
                            default: ((uint8_t *)gs.out[g])[q] = ((const uint8_t *)gs.col[g])[row]; break;
                            }
                        }
                    }
                    pos += __popc(bm[j]);
                }
            }
            excl += btot;
        }
        __syncthreads(); // mask words and indices free for the next round
    }
    if (lost) // let late copies land before the block's shared memory goes away (bounded)
        for (int st = 0; st < FT_STAGES && st < use; st++) {
            const long long u = use - 1 - ((use - 1 - st) % FT_STAGES); // last use of stage st
            mbar_wait(&s_bar[st], (uint32_t)(u / FT_STAGES) & 1u, limit);
        }
    if (b == G - 1 && threadIdx.x == 0) {
        *d_count = (long long)before;
        if ((long long)before > cap)
            set_status(d_status, TDP_ERR_CAPACITY);
    }
}

tdp_status make_gatherset(const tdp_col *cols, int32_t ncols, const int32_t *gather_cols, int32_t ngather,
                          void *const *gather_out, int64_t n, GatherSet *gs)
{
    if (ngather < 0 || ngather > TDP_MAX_GATHER || (ngather > 0 && (!gather_cols || !gather_out)))
        return TDP_ERR_INVALID_ARG;
    gs->n = ngather;
    for (int g = 0; g < TDP_MAX_GATHER; g++) {
        gs->col[g] = nullptr;
        gs->out[g] = nullptr;
        gs->size[g] = 0;
        gs->vec_ok[g] = 0;
    }
    for (int g = 0; g < ngather; g++) {
        int c = gather_cols[g];
        if (c < 0 || c >= ncols || cols[c].n < n || !gather_out[g])
            return TDP_ERR_INVALID_ARG;
        int sz = dtype_size(cols[c].dtype);
        if (sz == 0)
            return TDP_ERR_UNSUPPORTED_DTYPE;
        gs->col[g] = cols[c].data;
        gs->out[g] = gather_out[g];
        gs->size[g] = sz;
        gs->vec_ok[g] = ((uintptr_t)cols[c].data % 16) == 0;
    }
    return TDP_OK;
}

// Steps (4 rows a thread each) per tile for predicate columns taking
// `row_bytes` bytes a row: a stage of about 16 KiB.
static int filter_steps(int row_bytes)
{
    int steps = FT_MAX_STEPS;
    while (steps > 1 && (size_t)FT_THREADS * 4 * steps * row_bytes > 16 * 1024)
        steps >>= 1;
    return steps;
}

// Blocks of the cooperative launch: as many as fit on the GPU at once.
static int filter_grid_cap() { return 4 * num_sms(); }

template <int STEPS>
static tdp_status launch_filter(const PredSet &ps, const GatherSet &gs, long long n, const long long *d_n,
                                int32_t *out_rowid, long long cap, long long *d_count, void *ws, int32_t *d_status,
                                cudaStream_t s)
{
    constexpr long long TILE = FT_THREADS * 4 * STEPS;
    constexpr long long MASK_ROWS = (long long)FT_MASK_BYTES * 8;
    size_t pred_bytes = 0;
    for (int p = 0; p < ps.n; p++)
        pred_bytes += (size_t)TILE * dtype_size(ps.dt[p]);
    // a stage also holds one write batch of row ids (+ 3 for alignment)
    const uint32_t stage_bytes =
        (uint32_t)align_up(std::max<size_t>(pred_bytes, (size_t)(FT_WROWS + 4) * 4), 128);
    const size_t smem = (size_t)FT_STAGES * stage_bytes + FT_MASK_BYTES;
    auto kern = filter_kernel<STEPS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FT_THREADS, smem) != cudaSuccess || per_sm < 1)
        return TDP_ERR_CUDA;
    const long long tiles = (n + TILE - 1) / TILE;
    const int G = (int)std::min<long long>({tiles, (long long)per_sm * num_sms(), (long long)filter_grid_cap()});
    // rows per chunk: the table spread evenly over the blocks, in whole
    // tiles, at most what the mask of a chunk holds
    const long long per_block_tiles = (tiles + G - 1) / G;
    const long long chunk_rows = std::min(per_block_tiles * TILE, MASK_ROWS);
    const int rounds = (int)((n + (long long)G * chunk_rows - 1) / ((long long)G * chunk_rows));
    unsigned *barrier = (unsigned *)ws;
    unsigned long long *counts = (unsigned long long *)((char *)ws + 16);
    cudaMemsetAsync(ws, 0, 16, s);
    const uint32_t limit = spin_limit();
    void *args[] = {(void *)&ps, (void *)&gs, (void *)&n, (void *)&d_n, (void *)&out_rowid, (void *)&cap,
                    (void *)&d_count, (void *)&counts, (void *)&barrier, (void *)&d_status, (void *)&limit,
                    (void *)&stage_bytes, (void *)&chunk_rows, (void *)&rounds};
    if (cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(FT_THREADS), args, smem, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    return launch_status();
}

tdp_status filter_rows(const PredSet &ps, long long n, const long long *d_n, int32_t *out_rowid, long long cap,
                       long long *d_count, const GatherSet *gs, void *ws, int32_t *d_status, cudaStream_t s)
{
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(long long), s);
        return launch_status();
    }
    GatherSet none;
    none.n = 0;
    const GatherSet &g = gs ? *gs : none;
    int row_bytes = 0;
    for (int p = 0; p < ps.n; p++)
        row_bytes += dtype_size(ps.dt[p]);
    switch (filter_steps(row_bytes)) {
    case 8: return launch_filter<8>(ps, g, n, d_n, out_rowid, cap, d_count, ws, d_status, s);
    case 4: return launch_filter<4>(ps, g, n, d_n, out_rowid, cap, d_count, ws, d_status, s);
    case 2: return launch_filter<2>(ps, g, n, d_n, out_rowid, cap, d_count, ws, d_status, s);
    default: return launch_filter<1>(ps, g, n, d_n, out_rowid, cap, d_count, ws, d_status, s);
    }
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_filter_workspace(int64_t n)
{
    // barrier counter + one count per (round, block): at most one per tile
    // of the smallest size plus one per block
    long long tiles = (n + FT_MIN_TILE - 1) / FT_MIN_TILE;
    return align_up(16 + (size_t)(tiles + filter_grid_cap()) * 8, 256);
}

extern "C" tdp_status tdp_filter(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                                 int64_t n, const int64_t *d_n, int32_t *out_rowid, int64_t capacity,
                                 int64_t *d_count,
                                 const int32_t *gather_cols, int32_t ngather, void *const *gather_out, void *ws,
                                 size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || !d_count || capacity < 0 || (ncols > 0 && !cols))
        return TDP_ERR_INVALID_ARG;
    PredSet ps;
    tdp_status st = make_predset(cols, ncols, preds, npreds, n, &ps);
    if (st != TDP_OK)
        return st;
    GatherSet gs;
    st = make_gatherset(cols, ncols, gather_cols, ngather, gather_out, n, &gs);
    if (st != TDP_OK)
        return st;
    if (n > 0 && (ws_bytes < tdp_filter_workspace(n) || !ws))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (n > 0 && (uintptr_t)ws % 16)
        return TDP_ERR_INVALID_ARG;
    return filter_rows(ps, n, (const long long *)d_n, out_rowid, capacity, (long long *)d_count, &gs, ws, d_status,
                       (cudaStream_t)stream);
}
