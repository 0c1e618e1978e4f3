// K1/K2: predicate filter with stream compaction and fused column gather.
//
// One pass over the predicate columns; one tile of TILE = 256 x 4 x STEPS
// rows per block (16384 rows while the predicate columns take <= 4 bytes a
// row, fewer for wider predicates so that a tile stays <= 64 KiB).
//   1. Thread 0 stages the tile of every predicate column in shared memory
//      with one bulk copy per column (cp.async.bulk, completion on an
//      mbarrier); tiles at the ragged end, and columns whose base is not
//      16-byte aligned, are read with plain loads instead.
//   2. Lane l of warp w tests rows w*STEPS*128 + j*128 + 4l..4l+3 (step j):
//      every comparison is a range test (lo <= v <= hi) != neg on the
//      column's own type.  Ballots + popc give each row its rank within the
//      warp, the 8 warp totals its rank within the tile.
//   3. The qualifying row ids are written to shared memory (over the
//      consumed predicate tile) at their tile-local ranks, while warp 0 runs
//      the decoupled look-back over earlier tiles for the tile's output
//      offset (tiles are numbered by block index; every wait is bounded).
//   4. The block writes its run of row ids, and the gathered columns at those
//      rows, to consecutive output slots: coalesced stores.
// Output is stable (row order).
#include <algorithm>

#include "filter_api.cuh"

namespace tdp {

constexpr int FT_THREADS = 256;
constexpr int FT_MAX_STEPS = 16;
constexpr int FT_MIN_TILE = FT_THREADS * 4; // 1024 rows: the workspace is sized for this tile
constexpr int FT_SMEM_CAP = 64 * 1024;      // predicate bytes of one tile

// Same for rows read from global memory (ragged tile or unaligned column).
template <int STEPS>
__device__ __forceinline__ void ft_test_global(const PredSet &ps, int p, long long r0, long long n,
                                               unsigned (&m)[STEPS])
{
    const unsigned neg = (unsigned)ps.neg[p];
    const long long lo = ps.lo[p];
    const unsigned long long span = (unsigned long long)(ps.hi[p] - lo);
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        long long v[4];
        load4_int(ps.col[p], ps.dt[p], ps.vec_ok[p], r0 + j * 128, n, v);
        unsigned t = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
            t |= range_holds64(v[k], lo, span, neg) << k;
        m[j] &= t;
    }
}

template <int STEPS>
__global__ void __launch_bounds__(FT_THREADS, 3) filter_kernel(PredSet ps, GatherSet gs, long long n_host,
                                                            const long long *d_n, int32_t *out_rowid, long long cap,
                                                            long long *d_count, unsigned long long *tile_status,
                                                            int32_t *d_status, uint32_t limit, long long num_tiles)
{
    constexpr int TILE = FT_THREADS * 4 * STEPS;
    extern __shared__ __align__(128) unsigned char ft_smem[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned s_warp[FT_THREADS / 32];
    __shared__ unsigned long long s_excl;

    const long long tile = blockIdx.x;
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    const long long rbase = tile * TILE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lrow = warp * (STEPS * 128) + 4 * lane;

    // 1. stage the predicate columns of a full tile (all of them 16-byte aligned)
    bool bulk = ps.n > 0 && rbase + TILE <= n;
    for (int p = 0; p < ps.n; p++)
        bulk = bulk && ps.vec_ok[p];
    if (bulk && threadIdx.x == 0) {
        uint32_t bytes = 0;
        for (int p = 0; p < ps.n; p++)
            bytes += TILE * (uint32_t)dtype_size_dev(ps.dt[p]);
        mbar_init(&s_bar, 1);
        mbar_arrive_expect_tx(&s_bar, bytes);
        uint32_t off = 0;
        for (int p = 0; p < ps.n; p++) {
            const uint32_t sz = TILE * (uint32_t)dtype_size_dev(ps.dt[p]);
            bulk_load(ft_smem + off, (const char *)ps.col[p] + (size_t)rbase * dtype_size_dev(ps.dt[p]), sz, &s_bar);
            off += sz;
        }
    }
    __syncthreads(); // the mbarrier is initialised before anyone waits on it

    unsigned m[STEPS];
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        const long long r = rbase + lrow + j * 128;
        m[j] = r + 3 < n ? 0xfu : (r + 2 < n ? 0x7u : (r + 1 < n ? 0x3u : (r < n ? 0x1u : 0u)));
    }
    if (bulk) {
        const bool ok = mbar_wait(&s_bar, 0, limit);
        if (!ok)
            set_status(d_status, TDP_ERR_TIMEOUT);
        uint32_t off = 0;
        for (int p = 0; p < ps.n; p++) {
            pred_test_smem<STEPS>(ps, p, ft_smem + off, lrow, m);
            off += TILE * dtype_size_dev(ps.dt[p]);
        }
    } else {
        for (int p = 0; p < ps.n; p++)
            ft_test_global<STEPS>(ps, p, rbase + lrow, n, m);
    }

    // 2. ranks within the warp and the tile
    // per step: rank of the lane's first row within the step (low 16 bits) and
    // the step's count (high 16 bits)
    const unsigned lt = lanemask_lt();
    unsigned rank[STEPS], warp_tot = 0;
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        unsigned c = 0, pre = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            unsigned b = __ballot_sync(0xffffffffu, (m[j] >> k) & 1u);
            c += __popc(b);
            pre += __popc(b & lt);
        }
        rank[j] = c << 16 | pre;
        warp_tot += c;
    }
    if (lane == 0)
        s_warp[warp] = warp_tot;
    __syncthreads(); // predicate tile consumed; warp totals visible
    unsigned woff = 0, btot = 0;
#pragma unroll
    for (int w = 0; w < FT_THREADS / 32; w++) {
        unsigned t = s_warp[w];
        woff += w < warp ? t : 0;
        btot += t;
    }

    // 3. row ids to shared memory at their tile ranks; look-back for the tile offset
    int32_t *stage = (int32_t *)ft_smem;
    {
        unsigned pos = woff;
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            unsigned q = pos + (rank[j] & 0xffffu);
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (m[j] >> k & 1)
                    stage[q++] = (int32_t)(rbase + lrow + j * 128 + k);
            pos += rank[j] >> 16;
        }
    }
    if (warp == 0) {
        const unsigned long long e = lookback_exclusive(tile_status, tile, btot, limit, d_status);
        if (lane == 0) {
            s_excl = e;
            if (tile == num_tiles - 1) {
                const long long total = (long long)(e + btot);
                *d_count = total;
                if (total > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();

    // 4. coalesced output of the tile's run
    const long long excl = (long long)s_excl;
    const unsigned lim = (unsigned)max(0ll, min((long long)btot, cap - excl));
    if (out_rowid)
        for (unsigned i = threadIdx.x; i < lim; i += FT_THREADS)
            out_rowid[excl + i] = stage[i];
    for (int g = 0; g < gs.n; g++) {
        const void *col = gs.col[g];
        void *out = gs.out[g];
        switch (gs.size[g]) {
        case 8:
#pragma unroll 4
            for (unsigned i = threadIdx.x; i < lim; i += FT_THREADS)
                ((long long *)out)[excl + i] = __ldg((const long long *)col + stage[i]);
            break;
        case 4:
#pragma unroll 4
            for (unsigned i = threadIdx.x; i < lim; i += FT_THREADS)
                ((int32_t *)out)[excl + i] = __ldg((const int32_t *)col + stage[i]);
            break;
        case 2:
#pragma unroll 4
            for (unsigned i = threadIdx.x; i < lim; i += FT_THREADS)
                ((uint16_t *)out)[excl + i] = ((const uint16_t *)col)[stage[i]];
            break;
        default:
#pragma unroll 4
            for (unsigned i = threadIdx.x; i < lim; i += FT_THREADS)
                ((uint8_t *)out)[excl + i] = ((const uint8_t *)col)[stage[i]];
            break;
        }
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

// Rows per tile for predicate columns taking `row_bytes` bytes a row.
static int filter_steps(int row_bytes)
{
    int steps = FT_MAX_STEPS;
    while (steps > 1 && (size_t)FT_THREADS * 4 * steps * row_bytes > FT_SMEM_CAP)
        steps >>= 1;
    return steps;
}

template <int STEPS>
static tdp_status launch_filter(const PredSet &ps, const GatherSet &gs, long long n, const long long *d_n,
                                int32_t *out_rowid, long long cap, long long *d_count, void *ws, int32_t *d_status,
                                cudaStream_t s)
{
    constexpr long long TILE = FT_THREADS * 4 * STEPS;
    const long long tiles = (n + TILE - 1) / TILE;
    size_t pred_bytes = 0;
    for (int p = 0; p < ps.n; p++)
        pred_bytes += (size_t)TILE * dtype_size(ps.dt[p]);
    const size_t smem = std::max(pred_bytes, (size_t)TILE * 4);
    auto kern = filter_kernel<STEPS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    unsigned long long *status = (unsigned long long *)((char *)ws + 16);
    cudaMemsetAsync(status, 0, (size_t)tiles * 8, s);
    kern<<<(unsigned)tiles, FT_THREADS, smem, s>>>(ps, gs, n, d_n, out_rowid, cap, d_count, status, d_status,
                                                    spin_limit(), tiles);
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
    case 16: return launch_filter<16>(ps, g, n, d_n, out_rowid, cap, d_count, ws, d_status, s);
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
    // one look-back word per tile, sized for the smallest tile
    long long tiles = (n + FT_MIN_TILE - 1) / FT_MIN_TILE;
    return align_up(16 + (size_t)tiles * 8, 256);
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
    return filter_rows(ps, n, (const long long *)d_n, out_rowid, capacity, (long long *)d_count, &gs, ws, d_status,
                       (cudaStream_t)stream);
}
