// Group-by building blocks shared by tdp_groupby_agg and tdp_join_probe_agg.
#pragma once

#include "common.cuh"

namespace tdp {

// Key columns with their dense-domain encoding gid = sum_k (key_k - lo_k) * stride_k.
struct KeySet {
    const void *col[TDP_MAX_KEYS];
    int32_t dt[TDP_MAX_KEYS];
    int32_t vec_ok[TDP_MAX_KEYS];
    long long lo[TDP_MAX_KEYS];
    long long size[TDP_MAX_KEYS];
    long long stride[TDP_MAX_KEYS];
    int32_t n;
};

// Aggregates.  Accumulator slot 0 is COUNT(*); every other aggregate owns slot[a].
struct AggSet {
    const void *a[TDP_MAX_AGGS];
    int32_t adt[TDP_MAX_AGGS];
    int32_t avec[TDP_MAX_AGGS];
    const void *b[TDP_MAX_AGGS];
    int32_t bdt[TDP_MAX_AGGS];
    int32_t bvec[TDP_MAX_AGGS];
    long long k[TDP_MAX_AGGS];
    int32_t op[TDP_MAX_AGGS];
    int32_t slot[TDP_MAX_AGGS];
    int32_t n;
    int32_t nslots; // 1 + number of non-COUNT aggregates
    // The same aggregates indexed by accumulator slot (slot 0: COUNT), so that
    // kernels can loop over slots with compile-time indices.
    const void *sa[TDP_MAX_AGGS + 1];
    const void *sb[TDP_MAX_AGGS + 1];
    int32_t sadt[TDP_MAX_AGGS + 1];
    int32_t sbdt[TDP_MAX_AGGS + 1];
    long long sk[TDP_MAX_AGGS + 1];
    int32_t sop[TDP_MAX_AGGS + 1];
};

// Contribution of `row` to accumulator slot s (slot 0 counts rows).
__device__ __forceinline__ long long slot_value(const AggSet &as, int s, long long row)
{
    if (s == 0)
        return 1;
    long long va = load_int(as.sa[s], as.sadt[s], row);
    if (as.sop[s] == TDP_AGG_SUM_MUL_KMINUS)
        va *= as.sk[s] - load_int(as.sb[s], as.sbdt[s], row);
    return va;
}

tdp_status make_aggset(const tdp_col *cols, int32_t ncols, const tdp_agg *aggs, int32_t naggs, int64_t n,
                       AggSet *out);

// Initial value of an accumulator slot: 0 for COUNT/SUM, +max for MIN, -max for MAX.
__device__ __forceinline__ long long slot_init(const AggSet &as, int s)
{
    for (int a = 0; a < as.n; a++)
        if (as.slot[a] == s) {
            if (as.op[a] == TDP_AGG_MIN)
                return 0x7fffffffffffffffll;
            if (as.op[a] == TDP_AGG_MAX)
                return (long long)0x8000000000000000ull;
        }
    return 0;
}

// Contribution of one row to aggregate a (SUM_MUL_KMINUS: a*(k-b)).
__device__ __forceinline__ long long agg_value(const AggSet &as, int a, long long va, long long vb)
{
    return as.op[a] == TDP_AGG_SUM_MUL_KMINUS ? va * (as.k[a] - vb) : va;
}

// acc[slot] (+)= value with the aggregate's combine operator.
__device__ __forceinline__ void acc_update(long long *acc, int op, long long v)
{
    if (op == TDP_AGG_MIN)
        atomicMin(acc, v);
    else if (op == TDP_AGG_MAX)
        atomicMax(acc, v);
    else
        atomicAdd((unsigned long long *)acc, (unsigned long long)v);
}

// Combine operator of accumulator slot s.
__device__ __forceinline__ int slot_op(const AggSet &as, int s)
{
    for (int a = 0; a < as.n; a++)
        if (as.slot[a] == s && s != 0)
            return as.op[a];
    return TDP_AGG_SUM;
}

// Dense group id of `row`; false when a key lies outside its declared bounds.
__device__ __forceinline__ bool row_gid(const KeySet &ks, long long row, long long &gid)
{
    gid = 0;
    for (int k = 0; k < ks.n; k++) {
        long long v = load_int(ks.col[k], ks.dt[k], row) - ks.lo[k];
        if (v < 0 || v >= ks.size[k])
            return false;
        gid += v * ks.stride[k];
    }
    return true;
}

// Final value of aggregate a from its accumulator and the group count.
__device__ __forceinline__ long long agg_final(const AggSet &as, int a, const long long *acc)
{
    if (as.op[a] == TDP_AGG_COUNT)
        return acc[0];
    long long s = acc[as.slot[a]];
    if (as.op[a] == TDP_AGG_AVG) {
        long long c = acc[0];
        long long sg = s > 0 ? 1 : (s < 0 ? -1 : 0);
        return (2 * s + sg * c) / (2 * c);
    }
    return s;
}

// Dense-domain accumulator table: acc[gid * nslots + slot], slot 0 = count.
__global__ void dense_acc_init_kernel(AggSet as, long long D, long long *acc);

// Compacts the non-empty groups of a dense accumulator table in ascending gid
// order into the outputs (keys decoded from gid).  Tiles of 1024 gids with a
// decoupled look-back for the output offsets.
struct DenseOut {
    void *key_out[TDP_MAX_KEYS];
    int32_t key_dt[TDP_MAX_KEYS];
    long long *agg_out[TDP_MAX_AGGS];
};

tdp_status dense_finalize(const KeySet &ks, const AggSet &as, const DenseOut &out, long long D, const long long *acc,
                          long long capacity, int64_t *d_ngroups, void *ws, int32_t *d_status, cudaStream_t s);
size_t dense_finalize_ws(long long D);

} // namespace tdp
