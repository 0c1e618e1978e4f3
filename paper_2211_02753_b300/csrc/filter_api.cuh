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

} // namespace tdp
