// K1/K2: predicate filter with stream compaction and fused column gather.
//
// One pass over the predicate columns.  A tile is 256 threads x 16 rows.
// Warp w of a tile owns 512 consecutive rows, visited in 4 steps of 128 rows
// in which lane l holds rows 4l..4l+3 (one 16-byte load of an int32 column,
// a 4-byte load of an int8 column, two 16-byte loads of an int64 column, so
// each warp step reads one contiguous 512 B / 128 B / 1 KiB span).  Every
// row's output slot is found with warp ballots + popc (one ballot per row
// position within the lane's 4 rows), a scan over the 8 warps of the tile and
// a decoupled look-back over earlier tiles (tile ids from an atomic ticket,
// so every predecessor is already resident).  Output is stable.
#include "filter_api.cuh"

namespace tdp {

constexpr int FT_THREADS = 256;
constexpr int FT_STEPS = 4;
constexpr int FT_WARP_ROWS = FT_STEPS * 128;
constexpr int FT_TILE = FT_THREADS / 32 * FT_WARP_ROWS; // 4096

// Copies element k (0..3) of a 4-row group at row r of a column of `size`
// bytes to out[pos].
__device__ __forceinline__ void gather_store(const void *col, void *out, int size, bool vec_ok, long long r,
                                             long long n, unsigned m4, long long pos, long long cap)
{
    if (size == 8) {
        long long v[4];
        if (vec_ok && r + 3 < n) {
            longlong2 a = __ldg((const longlong2 *)((const long long *)col + r));
            longlong2 b = __ldg((const longlong2 *)((const long long *)col + r + 2));
            v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                v[k] = (m4 >> k & 1) ? ((const long long *)col)[r + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m4 >> k & 1) {
                if (pos < cap)
                    ((long long *)out)[pos] = v[k];
                pos++;
            }
    } else if (size == 4) {
        int v[4];
        if (vec_ok && r + 3 < n) {
            int4 a = __ldg((const int4 *)((const int *)col + r));
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                v[k] = (m4 >> k & 1) ? ((const int *)col)[r + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m4 >> k & 1) {
                if (pos < cap)
                    ((int *)out)[pos] = v[k];
                pos++;
            }
    } else if (size == 2) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m4 >> k & 1) {
                if (pos < cap)
                    ((uint16_t *)out)[pos] = ((const uint16_t *)col)[r + k];
                pos++;
            }
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m4 >> k & 1) {
                if (pos < cap)
                    ((uint8_t *)out)[pos] = ((const uint8_t *)col)[r + k];
                pos++;
            }
    }
}

__global__ void __launch_bounds__(FT_THREADS) filter_kernel(PredSet ps, GatherSet gs, long long n_host,
                                                            const long long *d_n, int32_t *out_rowid, long long cap, long long *d_count,
                                                            unsigned long long *tile_status, unsigned *ticket,
                                                            int32_t *d_status, uint32_t limit, long long num_tiles)
{
    // The block takes a ticket; warp w then owns sub-tile ticket*8 + w and does
    // its own decoupled look-back (no block-wide barrier after the start).
    __shared__ long long s_tile;

    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long wtile = tile * (FT_THREADS / 32) + warp;
    const long long r0 = tile * FT_TILE + (long long)warp * FT_WARP_ROWS + 4 * lane;

    unsigned m[FT_STEPS];
#pragma unroll
    for (int j = 0; j < FT_STEPS; j++) {
        long long r = r0 + j * 128;
        m[j] = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
            m[j] |= (r + k < n) ? (1u << k) : 0u;
    }
    for (int p = 0; p < ps.n; p++) {
        long long v[FT_STEPS][4];
        load_rows<FT_STEPS>(ps.col[p], ps.dt[p], ps.vec_ok[p], r0, n, v);
#pragma unroll
        for (int j = 0; j < FT_STEPS; j++)
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (!cmp_holds(v[j][k], ps.cmp[p], ps.lit[p]))
                    m[j] &= ~(1u << k);
    }

    // ballot / popc ranks
    const unsigned lt = lanemask_lt();
    unsigned step_cnt[FT_STEPS], lane_pref[FT_STEPS];
    unsigned warp_tot = 0;
#pragma unroll
    for (int j = 0; j < FT_STEPS; j++) {
        unsigned c = 0, pre = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            unsigned b = __ballot_sync(0xffffffffu, (m[j] >> k) & 1u);
            c += __popc(b);
            pre += __popc(b & lt);
        }
        step_cnt[j] = c;
        lane_pref[j] = pre;
        warp_tot += c;
    }
    const unsigned long long excl = lookback_exclusive(tile_status, wtile, warp_tot, limit, d_status);
    if (lane == 0 && wtile == num_tiles - 1) { // num_tiles counts warp sub-tiles
        long long total = (long long)(excl + warp_tot);
        *d_count = total;
        if (total > cap)
            set_status(d_status, TDP_ERR_CAPACITY);
    }

    long long pos = (long long)excl;
#pragma unroll
    for (int j = 0; j < FT_STEPS; j++) {
        const long long r = r0 + j * 128;
        long long p = pos + lane_pref[j];
        if (m[j]) {
            if (out_rowid) {
                long long q = p;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (m[j] >> k & 1) {
                        if (q < cap)
                            out_rowid[q] = (int32_t)(r + k);
                        q++;
                    }
            }
            for (int g = 0; g < gs.n; g++)
                gather_store(gs.col[g], gs.out[g], gs.size[g], gs.vec_ok[g], r, n, m[j], p, cap);
        }
        pos += step_cnt[j];
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

tdp_status filter_rows(const PredSet &ps, long long n, const long long *d_n, int32_t *out_rowid, long long cap,
                       long long *d_count, const GatherSet *gs, void *ws, int32_t *d_status, cudaStream_t s)
{
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(long long), s);
        return launch_status();
    }
    GatherSet none;
    none.n = 0;
    long long tiles = (n + FT_TILE - 1) / FT_TILE;
    long long wtiles = tiles * (FT_THREADS / 32); // one look-back word per warp sub-tile
    unsigned *ticket = (unsigned *)ws;
    unsigned long long *status = (unsigned long long *)((char *)ws + 16);
    cudaMemsetAsync(ws, 0, 16 + (size_t)wtiles * 8, s);
    filter_kernel<<<(unsigned)tiles, FT_THREADS, 0, s>>>(ps, gs ? *gs : none, n, d_n, out_rowid, cap, d_count, status,
                                                         ticket, d_status, spin_limit(), wtiles);
    return launch_status();
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_filter_workspace(int64_t n)
{
    long long wtiles = (n + FT_TILE - 1) / FT_TILE * (FT_THREADS / 32);
    return align_up(16 + (size_t)wtiles * 8, 256);
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
