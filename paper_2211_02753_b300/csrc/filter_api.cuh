// Internal entry of the filter kernel (filter.cu) for other operators.
#pragma once

#include "common.cuh"

namespace tdp {

struct GatherSet {
    const void *col[TDP_MAX_GATHER];
    void *out[TDP_MAX_GATHER];
    int32_t size[TDP_MAX_GATHER]; // element bytes: 1, 2, 4 or 8
    int32_t vec_ok[TDP_MAX_GATHER];
    int32_t n;
};

tdp_status make_gatherset(const tdp_col *cols, int32_t ncols, const int32_t *gather_cols, int32_t ngather,
                          void *const *gather_out, int64_t n, GatherSet *gs);

// Compacts the ids of rows 0..n-1 (0..min(n,*d_n)-1 if d_n) that satisfy `ps` into out_rowid (stable),
// count to *d_count; optional fused gather.  ws: tdp_filter_workspace(n).
tdp_status filter_rows(const PredSet &ps, long long n, const long long *d_n, int32_t *out_rowid, long long cap,
                       long long *d_count, const GatherSet *gs, void *ws, int32_t *d_status, cudaStream_t s);

// Clears the mask bits (4 per step) of rows that fail predicate p.  The
// tile of the predicate's column is in shared memory at tile_col; lane rows
// are lrow + j*128 + 0..3 for step j (tile-local).
template <int STEPS>
__device__ __forceinline__ void pred_test_smem(const PredSet &ps, int p, const unsigned char *tile_col, int lrow,
                                             unsigned (&m)[STEPS])
{
    const int dt = ps.dt[p];
    const unsigned neg = (unsigned)ps.neg[p];
    if (dt == TDP_I64) {
        const long long lo = ps.lo[p];
        const unsigned long long span = (unsigned long long)(ps.hi[p] - lo);
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            const longlong2 *q = (const longlong2 *)(tile_col + (size_t)(lrow + j * 128) * 8);
            longlong2 a = q[0], b = q[1];
            unsigned t = range_holds64(a.x, lo, span, neg) | range_holds64(a.y, lo, span, neg) << 1 |
                         range_holds64(b.x, lo, span, neg) << 2 | range_holds64(b.y, lo, span, neg) << 3;
            m[j] &= t;
        }
        return;
    }
    const int lo = (int)ps.lo[p];
    const unsigned span = (unsigned)((int)ps.hi[p] - lo);
    if (dt == TDP_I32) {
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            int4 w = *(const int4 *)(tile_col + (size_t)(lrow + j * 128) * 4);
            unsigned t = range_holds32(w.x, lo, span, neg) | range_holds32(w.y, lo, span, neg) << 1 |
                         range_holds32(w.z, lo, span, neg) << 2 | range_holds32(w.w, lo, span, neg) << 3;
            m[j] &= t;
        }
        return;
    }
    const bool sgn = dt == TDP_I8;
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        unsigned w = *(const unsigned *)(tile_col + lrow + j * 128);
        unsigned t = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            unsigned b = (w >> (8 * k)) & 0xffu;
            int v = sgn ? (int)(int8_t)b : (int)b;
            t |= range_holds32(v, lo, span, neg) << k;
        }
        m[j] &= t;
    }
}

} // namespace tdp
