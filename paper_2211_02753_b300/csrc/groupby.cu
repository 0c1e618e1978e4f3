// K5 (small-domain group-by) and the entry point tdp_groupby_agg.
//
// SMALL_DOMAIN: when every key column carries bounds (the column metadata of
// Sec. 2 that picks an operator strategy) the key tuple maps to a dense group
// id gid = sum_k (key_k - lo_k) * stride_k.  One pass over the rows (fused
// with the WHERE predicates) adds every row into a private copy of the dense
// accumulator table: one copy per warp when the table is tiny (a handful of
// groups, e.g. flag x status), one per block when it fits in shared memory,
// else the global table itself.  Copies are merged into the global table
// with 64-bit atomics (integer sums are exact, so the result does not depend
// on the order), and a compaction kernel emits the non-empty groups in
// ascending gid order, which is ascending key order.
//
// SORT: see groupby_sort.cu.  PARTITION (bounded keys, domain too large for
// one shared-memory table): see groupby_part.cu.
#include "groupby.cuh"

namespace tdp {

tdp_status make_aggset(const tdp_col *cols, int32_t ncols, const tdp_agg *aggs, int32_t naggs, int64_t n,
                       AggSet *as)
{
    if (naggs < 1 || naggs > TDP_MAX_AGGS || !aggs)
        return TDP_ERR_INVALID_ARG;
    as->n = naggs;
    as->nslots = 1;
    for (int a = 0; a < TDP_MAX_AGGS; a++) {
        as->a[a] = as->b[a] = nullptr;
        as->adt[a] = as->bdt[a] = TDP_I64;
        as->avec[a] = as->bvec[a] = 0;
        as->k[a] = 0;
        as->op[a] = 0;
        as->slot[a] = 0;
    }
    for (int a = 0; a < naggs; a++) {
        const tdp_agg &g = aggs[a];
        if (g.op < TDP_AGG_COUNT || g.op > TDP_AGG_MAX)
            return TDP_ERR_INVALID_ARG;
        as->op[a] = g.op;
        as->k[a] = g.k;
        if (g.op == TDP_AGG_COUNT) {
            as->slot[a] = 0;
            continue;
        }
        if (g.a < 0 || g.a >= ncols || cols[g.a].n < n)
            return TDP_ERR_INVALID_ARG;
        if (!is_int_dtype(cols[g.a].dtype))
            return TDP_ERR_UNSUPPORTED_DTYPE;
        as->a[a] = cols[g.a].data;
        as->adt[a] = cols[g.a].dtype;
        as->avec[a] = ((uintptr_t)cols[g.a].data % 16) == 0;
        if (g.op == TDP_AGG_SUM_MUL_KMINUS) {
            if (g.b < 0 || g.b >= ncols || cols[g.b].n < n)
                return TDP_ERR_INVALID_ARG;
            if (!is_int_dtype(cols[g.b].dtype))
                return TDP_ERR_UNSUPPORTED_DTYPE;
            as->b[a] = cols[g.b].data;
            as->bdt[a] = cols[g.b].dtype;
            as->bvec[a] = ((uintptr_t)cols[g.b].data % 16) == 0;
        }
        as->slot[a] = as->nslots++;
    }
    for (int s = 0; s <= TDP_MAX_AGGS; s++) {
        as->sa[s] = as->sb[s] = nullptr;
        as->sadt[s] = as->sbdt[s] = TDP_I64;
        as->sk[s] = 0;
        as->sop[s] = TDP_AGG_COUNT;
    }
    for (int a = 0; a < naggs; a++) {
        int s = as->slot[a];
        if (s == 0)
            continue;
        as->sa[s] = as->a[a];
        as->sb[s] = as->b[a];
        as->sadt[s] = as->adt[a];
        as->sbdt[s] = as->bdt[a];
        as->sk[s] = as->k[a];
        as->sop[s] = as->op[a];
    }
    return TDP_OK;
}

__global__ void dense_acc_init_kernel(AggSet as, long long D, long long *acc)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = D * as.nslots;
    for (; e < total; e += (long long)gridDim.x * blockDim.x)
        acc[e] = slot_init(as, (int)(e % as.nslots));
}

constexpr int SD_THREADS = 256;

template <bool SEL>
__global__ void __launch_bounds__(SD_THREADS) small_domain_kernel(PredSet ps, KeySet ks, AggSet as, long long n,
                                                                  const int32_t *sel, const long long *d_nsel,
                                                                  long long D, int copies, long long *gacc,
                                                                  int32_t *d_status)
{
    extern __shared__ long long sacc[];
    const int NS = as.nslots;
    const long long tab = D * NS;
    if (copies > 0) {
        for (long long e = threadIdx.x; e < tab * copies; e += SD_THREADS)
            sacc[e] = slot_init(as, (int)(e % NS));
        __syncthreads();
    }
    long long *my = copies == 0 ? gacc : sacc + (copies == 1 ? 0 : (long long)(threadIdx.x >> 5) * tab);
    bool bad = false;
    if (!SEL) {
        if (d_nsel)
            n = min(*d_nsel, n);
        const long long stride = (long long)gridDim.x * SD_THREADS * 4;
        for (long long r = ((long long)blockIdx.x * SD_THREADS + threadIdx.x) * 4; r < n; r += stride) {
            unsigned m = eval_preds4(ps, r, n);
            if (!m)
                continue;
            long long gid[4] = {0, 0, 0, 0};
            for (int k = 0; k < ks.n; k++) {
                long long v[4];
                load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, n, v);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    long long d = v[j] - ks.lo[k];
                    if ((m >> j & 1) && (d < 0 || d >= ks.size[k])) {
                        m &= ~(1u << j);
                        bad = true;
                    }
                    gid[j] += d * ks.stride[k];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (m >> j & 1)
                    atomicAdd((unsigned long long *)&my[gid[j] * NS], 1ull);
            for (int a = 0; a < as.n; a++) {
                if (as.op[a] == TDP_AGG_COUNT)
                    continue;
                long long va[4], vb[4] = {0, 0, 0, 0};
                load4_int(as.a[a], as.adt[a], as.avec[a], r, n, va);
                if (as.op[a] == TDP_AGG_SUM_MUL_KMINUS)
                    load4_int(as.b[a], as.bdt[a], as.bvec[a], r, n, vb);
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (m >> j & 1)
                        acc_update(&my[gid[j] * NS + as.slot[a]], as.op[a], agg_value(as, a, va[j], vb[j]));
            }
        }
    } else {
        long long nsel = min(*d_nsel, n);
        for (long long i = (long long)blockIdx.x * SD_THREADS + threadIdx.x; i < nsel;
             i += (long long)gridDim.x * SD_THREADS) {
            long long row = sel[i];
            if (!eval_preds1(ps, row))
                continue;
            long long gid;
            if (!row_gid(ks, row, gid)) {
                bad = true;
                continue;
            }
            atomicAdd((unsigned long long *)&my[gid * NS], 1ull);
            for (int a = 0; a < as.n; a++) {
                if (as.op[a] == TDP_AGG_COUNT)
                    continue;
                long long va = load_int(as.a[a], as.adt[a], row);
                long long vb = as.op[a] == TDP_AGG_SUM_MUL_KMINUS ? load_int(as.b[a], as.bdt[a], row) : 0;
                acc_update(&my[gid * NS + as.slot[a]], as.op[a], agg_value(as, a, va, vb));
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    if (copies > 0) {
        __syncthreads();
        for (long long e = threadIdx.x; e < tab; e += SD_THREADS) {
            int s = (int)(e % NS);
            int op = slot_op(as, s);
            long long init = slot_init(as, s);
            long long v = sacc[e];
            for (int c = 1; c < copies; c++) {
                long long u = sacc[c * tab + e];
                v = op == TDP_AGG_MIN ? min(v, u) : op == TDP_AGG_MAX ? max(v, u) : v + u;
            }
            if (v != init)
                acc_update(&gacc[e], op, v);
        }
    }
}

// Small domains (D * nslots <= SP_MAX_TAB accumulators): every thread owns a
// private slice of D x nslots accumulators in shared memory (odd 64-bit
// pitch, so that the lanes' slices fall on distinct banks), updated with
// plain loads and stores -- no atomics and no contention however few the
// groups are.  The block then folds its 256 slices (tree over threads in a
// fixed order) and adds each group's totals to the global accumulators.
constexpr int SP_MAX_TAB = 63;

__global__ void __launch_bounds__(SD_THREADS) small_domain_priv_kernel(PredSet ps, KeySet ks, AggSet as, long long n,
                                                                       const long long *d_nsel, int D, int pitch,
                                                                       long long *gacc, int32_t *d_status)
{
    extern __shared__ long long spriv[];
    const int NS = as.nslots;
    const int tab = D * NS;
    long long *my = spriv + (size_t)threadIdx.x * pitch;
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    __shared__ int s_op[TDP_MAX_AGGS + 1];
    if (threadIdx.x <= TDP_MAX_AGGS) {
        s_init[threadIdx.x] = threadIdx.x < NS ? slot_init(as, threadIdx.x) : 0;
        s_op[threadIdx.x] = threadIdx.x < NS ? slot_op(as, threadIdx.x) : TDP_AGG_SUM;
    }
    __syncthreads();
    for (int e = 0; e < tab; e++)
        my[e] = s_init[e % NS];
    bool bad = false;
    if (d_nsel)
        n = min(*d_nsel, n);
    const long long stride = (long long)gridDim.x * SD_THREADS * 4;
    for (long long r = ((long long)blockIdx.x * SD_THREADS + threadIdx.x) * 4; r < n; r += stride) {
        unsigned m = eval_preds4(ps, r, n);
        if (!m)
            continue;
        long long gid[4] = {0, 0, 0, 0};
        for (int k = 0; k < ks.n; k++) {
            long long v[4];
            load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, n, v);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const long long d = v[j] - ks.lo[k];
                if ((m >> j & 1) && (d < 0 || d >= ks.size[k])) {
                    m &= ~(1u << j);
                    bad = true;
                }
                gid[j] += d * ks.stride[k];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (m >> j & 1)
                my[gid[j] * NS] += 1;
        for (int sl = 1; sl < NS; sl++) {
            long long va[4], vb[4] = {0, 0, 0, 0};
            load4_int(as.sa[sl], as.sadt[sl], ((uintptr_t)as.sa[sl] % 16) == 0, r, n, va);
            const int op = s_op[sl];
            if (op == TDP_AGG_SUM_MUL_KMINUS)
                load4_int(as.sb[sl], as.sbdt[sl], ((uintptr_t)as.sb[sl] % 16) == 0, r, n, vb);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (!(m >> j & 1))
                    continue;
                long long *a = my + gid[j] * NS + sl;
                if (op == TDP_AGG_MIN)
                    *a = min(*a, va[j]);
                else if (op == TDP_AGG_MAX)
                    *a = max(*a, va[j]);
                else
                    *a += op == TDP_AGG_SUM_MUL_KMINUS ? va[j] * (as.sk[sl] - vb[j]) : va[j];
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    // fold the slices: tree over threads, then one global update per accumulator
    for (int h = SD_THREADS / 2; h > 0; h >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < h) {
            const long long *o = spriv + (size_t)(threadIdx.x + h) * pitch;
            for (int e = 0; e < tab; e++) {
                const int op = s_op[e % NS];
                my[e] = op == TDP_AGG_MIN ? min(my[e], o[e]) : op == TDP_AGG_MAX ? max(my[e], o[e]) : my[e] + o[e];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tab; e += SD_THREADS)
        if (spriv[e] != s_init[e % NS])
            acc_update(&gacc[e], s_op[e % NS], spriv[e]);
}

// The same private-slice scheme with the slot count NSX a compile-time
// constant and at most one a * (k - b) slot: MS is that slot (0 for none)
// when every slot combines by addition (ADD), else MS = -1 and the slot is
// the argument mslot.  Predicates are tested in their closed-range form (lo,
// hi and neg of the PredSet, clamped into the column's type, so a 64-bit
// unsigned distance decides every type); the first predicate's column is
// loaded one quad ahead, and once a quad's predicates are known the first
// two key columns and every value column of its four rows are loaded before
// any of them is used: one round trip to memory per quad instead of one per
// slot.  The slice offsets, and for ADD the per-slot arithmetic, are fixed
// at compile time.  Three blocks of 256 threads per SM (the shared slices
// allow three; the register cap keeps them resident).
template <int NSX, bool ADD, int MS>
__global__ void __launch_bounds__(SD_THREADS, 3) small_domain_priv_n_kernel(PredSet ps, KeySet ks, AggSet as, long long n,
                                                                            const long long *d_nsel, int D, int pitch,
                                                                            int mslot, long long *gacc,
                                                                            int32_t *d_status)
{
    constexpr int KB = TDP_MAX_KEYS < 2 ? TDP_MAX_KEYS : 2; // key columns loaded with the values
    extern __shared__ long long spriv[];
    const int tab = D * NSX;
    long long *my = spriv + (size_t)threadIdx.x * pitch;
    __shared__ long long s_init[NSX];
    __shared__ int s_op[NSX];
    if (threadIdx.x < NSX) {
        s_init[threadIdx.x] = slot_init(as, threadIdx.x);
        s_op[threadIdx.x] = slot_op(as, threadIdx.x);
    }
    __syncthreads();
    for (int e = 0; e < tab; e++)
        my[e] = s_init[e % NSX];
    if (MS >= 0)
        mslot = MS;
    int op[NSX];
    bool va_vec[NSX], is_mul[NSX];
#pragma unroll
    for (int sl = 1; sl < NSX; sl++) {
        op[sl] = s_op[sl];
        va_vec[sl] = ((uintptr_t)as.sa[sl] % 16) == 0;
        is_mul[sl] = MS >= 0 ? sl == MS : sl == mslot;
    }
    const void *bcol = mslot ? as.sb[mslot] : nullptr;
    const int bdt = mslot ? as.sbdt[mslot] : TDP_I64;
    const bool b_vec = mslot && ((uintptr_t)bcol % 16) == 0;
    const long long bk = mslot ? as.sk[mslot] : 0;
    bool bad = false;
    if (d_nsel)
        n = min(*d_nsel, n);
    const long long stride = (long long)gridDim.x * SD_THREADS * 4;
    // the first predicate's column of the thread's next quad is loaded one
    // iteration ahead (its values decide which rows the other loads serve)
    const bool pf = ps.n > 0;
    const long long p0lo = pf ? ps.lo[0] : 0;
    const unsigned long long p0span = pf ? (unsigned long long)ps.hi[0] - (unsigned long long)p0lo : 0;
    const unsigned p0neg = pf ? (unsigned)ps.neg[0] : 0u;
    long long r = ((long long)blockIdx.x * SD_THREADS + threadIdx.x) * 4;
    long long pv[4] = {0, 0, 0, 0};
    if (pf && r < n)
        load4_int(ps.col[0], ps.dt[0], ps.vec_ok[0], r, n, pv);
    for (; r < n; r += stride) {
        unsigned m = r + 3 < n ? 0xfu : (r + 2 < n ? 0x7u : (r + 1 < n ? 0x3u : 0x1u));
        if (pf) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                m &= ~((range_holds64(pv[k], p0lo, p0span, p0neg) ^ 1u) << k);
            if (r + stride < n)
                load4_int(ps.col[0], ps.dt[0], ps.vec_ok[0], r + stride, n, pv);
        }
        for (int p = 1; p < ps.n; p++) {
            long long v[4];
            load4_int(ps.col[p], ps.dt[p], ps.vec_ok[p], r, n, v);
            const long long lo = ps.lo[p];
            const unsigned long long span = (unsigned long long)ps.hi[p] - (unsigned long long)lo;
            const unsigned neg = (unsigned)ps.neg[p];
#pragma unroll
            for (int k = 0; k < 4; k++)
                m &= ~((range_holds64(v[k], lo, span, neg) ^ 1u) << k);
        }
        if (!m)
            continue;
        long long kv[KB][4];
#pragma unroll
        for (int k = 0; k < KB; k++)
            if (k < ks.n)
                load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, n, kv[k]);
        long long va[NSX][4], vb[4];
#pragma unroll
        for (int sl = 1; sl < NSX; sl++)
            load4_int(as.sa[sl], as.sadt[sl], va_vec[sl], r, n, va[sl]);
        if (mslot)
            load4_int(bcol, bdt, b_vec, r, n, vb);
        unsigned gid[4] = {0u, 0u, 0u, 0u}; // < D <= SP_MAX_TAB for the rows whose keys are in bounds
        auto add_key = [&](int k, const long long *v) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const long long d = v[j] - ks.lo[k];
                if ((m >> j & 1) && (unsigned long long)d >= (unsigned long long)ks.size[k]) {
                    m &= ~(1u << j);
                    bad = true;
                }
                gid[j] += (unsigned)d * (unsigned)ks.stride[k]; // wraps harmlessly for masked rows
            }
        };
#pragma unroll
        for (int k = 0; k < KB; k++)
            if (k < ks.n)
                add_key(k, kv[k]);
        for (int k = KB; k < ks.n; k++) {
            long long v[4];
            load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, n, v);
            add_key(k, v);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (!(m >> j & 1))
                continue;
            long long *a = my + gid[j] * NSX;
            a[0] += 1;
#pragma unroll
            for (int sl = 1; sl < NSX; sl++) {
                long long v;
                if (MS >= 0)
                    v = sl == MS ? va[sl][j] * (bk - vb[j]) : va[sl][j];
                else
                    v = is_mul[sl] ? va[sl][j] * (bk - vb[j]) : va[sl][j];
                if (ADD)
                    a[sl] += v;
                else
                    a[sl] = op[sl] == TDP_AGG_MIN ? min(a[sl], v) : op[sl] == TDP_AGG_MAX ? max(a[sl], v) : a[sl] + v;
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    for (int h = SD_THREADS / 2; h > 0; h >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < h) {
            const long long *o = spriv + (size_t)(threadIdx.x + h) * pitch;
            for (int e = 0; e < tab; e++) {
                const int sop = s_op[e % NSX];
                my[e] = sop == TDP_AGG_MIN ? min(my[e], o[e]) : sop == TDP_AGG_MAX ? max(my[e], o[e]) : my[e] + o[e];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tab; e += SD_THREADS)
        if (spriv[e] != s_init[e % NSX])
            acc_update(&gacc[e], s_op[e % NSX], spriv[e]);
}

constexpr int FIN_THREADS = 256;
constexpr int FIN_TILE = FIN_THREADS * 4;

__global__ void __launch_bounds__(FIN_THREADS) dense_finalize_kernel(KeySet ks, AggSet as, DenseOut out, long long D,
                                                                     const long long *acc, long long cap,
                                                                     long long *d_ngroups,
                                                                     unsigned long long *tile_status,
                                                                     unsigned *ticket, int32_t *d_status,
                                                                     uint32_t limit, long long ntiles)
{
    __shared__ long long s_tile;
    __shared__ unsigned s_warp[FIN_THREADS / 32];
    __shared__ unsigned long long s_excl;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const int NS = as.nslots;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g0 = tile * FIN_TILE + 4ll * threadIdx.x;
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 4; j++)
        if (g0 + j < D && acc[(g0 + j) * NS] > 0)
            m |= 1u << j;
    unsigned c = __popc(m), incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned t = lane < FIN_THREADS / 32 ? s_warp[lane] : 0, wi = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += u;
        }
        unsigned long long agg = __shfl_sync(0xffffffffu, wi, 31);
        if (lane < FIN_THREADS / 32)
            s_warp[lane] = wi - t; // exclusive warp offsets
        unsigned long long excl = lookback_exclusive(tile_status, tile, agg, limit, d_status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == ntiles - 1) {
                *d_ngroups = (long long)(excl + agg);
                if ((long long)(excl + agg) > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    long long pos = (long long)s_excl + s_warp[warp] + (incl - c);
    for (int j = 0; j < 4; j++) {
        if (!(m >> j & 1))
            continue;
        long long g = g0 + j;
        if (pos < cap) {
            for (int k = 0; k < ks.n; k++) {
                long long key = ks.lo[k] + (g / ks.stride[k]) % ks.size[k];
                switch (out.key_dt[k]) {
                case TDP_I8: ((int8_t *)out.key_out[k])[pos] = (int8_t)key; break;
                case TDP_U8: ((uint8_t *)out.key_out[k])[pos] = (uint8_t)key; break;
                case TDP_I32: ((int32_t *)out.key_out[k])[pos] = (int32_t)key; break;
                default: ((long long *)out.key_out[k])[pos] = key; break;
                }
            }
            for (int a = 0; a < as.n; a++)
                out.agg_out[a][pos] = agg_final(as, a, acc + g * NS);
        }
        pos++;
    }
}

size_t dense_finalize_ws(long long D)
{
    long long tiles = (D + FIN_TILE - 1) / FIN_TILE;
    return align_up(16 + (size_t)tiles * 8, 256);
}

tdp_status dense_finalize(const KeySet &ks, const AggSet &as, const DenseOut &out, long long D, const long long *acc,
                          long long capacity, int64_t *d_ngroups, void *ws, int32_t *d_status, cudaStream_t s)
{
    long long tiles = (D + FIN_TILE - 1) / FIN_TILE;
    cudaMemsetAsync(ws, 0, 16 + (size_t)tiles * 8, s);
    dense_finalize_kernel<<<(unsigned)tiles, FIN_THREADS, 0, s>>>(
        ks, as, out, D, acc, capacity, (long long *)d_ngroups, (unsigned long long *)((char *)ws + 16),
        (unsigned *)ws, d_status, spin_limit(), tiles);
    return launch_status();
}

// ------------------------------------------------------------------ host

tdp_status make_keyset(const tdp_col *cols, int32_t ncols, const int32_t *key_cols, int32_t nkeys, int64_t n,
                       KeySet *ks, bool need_bounds, long long *domain)
{
    if (nkeys < 1 || nkeys > TDP_MAX_KEYS || !key_cols)
        return TDP_ERR_INVALID_ARG;
    ks->n = nkeys;
    long long D = 1;
    for (int k = nkeys - 1; k >= 0; k--) {
        int c = key_cols[k];
        if (c < 0 || c >= ncols || cols[c].n < n)
            return TDP_ERR_INVALID_ARG;
        if (!is_int_dtype(cols[c].dtype))
            return TDP_ERR_UNSUPPORTED_DTYPE;
        ks->col[k] = cols[c].data;
        ks->dt[k] = cols[c].dtype;
        ks->vec_ok[k] = ((uintptr_t)cols[c].data % 16) == 0;
        if (cols[c].has_bounds && cols[c].hi >= cols[c].lo) {
            ks->lo[k] = cols[c].lo;
            ks->size[k] = cols[c].hi - cols[c].lo + 1;
        } else {
            if (need_bounds)
                return TDP_ERR_INVALID_ARG;
            ks->lo[k] = 0;
            ks->size[k] = 0;
        }
        ks->stride[k] = D;
        if (ks->size[k] > 0 && D <= (1ll << 40))
            D *= ks->size[k];
        else
            D = 1ll << 41;
    }
    for (int k = nkeys; k < TDP_MAX_KEYS; k++) {
        ks->col[k] = nullptr;
        ks->dt[k] = 0;
        ks->vec_ok[k] = 0;
        ks->lo[k] = ks->size[k] = ks->stride[k] = 0;
    }
    *domain = D;
    return TDP_OK;
}

static const long long SMALL_DOMAIN_MAX = 1ll << 22;

static bool keys_small_desc(const tdp_col *keys, int32_t nkeys, long long *D)
{
    long long d = 1;
    for (int k = 0; k < nkeys; k++) {
        if (!keys[k].has_bounds || keys[k].hi < keys[k].lo)
            return false;
        long long sz = keys[k].hi - keys[k].lo + 1;
        if (sz > SMALL_DOMAIN_MAX || d * sz > SMALL_DOMAIN_MAX)
            return false;
        d *= sz;
    }
    *D = d;
    return true;
}

int small_domain_copies(long long D, int nslots, size_t *smem)
{
    size_t tab = (size_t)D * nslots * 8;
    if (tab * (SD_THREADS / 32) <= 32 * 1024) {
        *smem = tab * (SD_THREADS / 32);
        return SD_THREADS / 32;
    }
    if (tab <= 160 * 1024) {
        *smem = tab;
        return 1;
    }
    *smem = 0;
    return 0;
}

size_t small_domain_ws(long long D, int naggs)
{
    return align_up((size_t)D * (1 + naggs) * 8, 256) + dense_finalize_ws(D);
}

tdp_status small_domain_run(const PredSet &ps, const KeySet &ks, const AggSet &as, long long D, long long n,
                            const int32_t *sel, const int64_t *d_nsel, const DenseOut &out, long long capacity,
                            int64_t *d_ngroups, void *ws, int32_t *d_status, cudaStream_t s)
{
    long long *acc = (long long *)ws;
    void *fin_ws = (char *)ws + align_up((size_t)D * as.nslots * 8, 256);
    dense_acc_init_kernel<<<(unsigned)std::min<long long>((D * as.nslots + 255) / 256, 4096), 256, 0, s>>>(as, D,
                                                                                                         acc);
    if (!sel && D * as.nslots <= SP_MAX_TAB) {
        // private per-thread accumulators
        const int pitch = (int)(D * as.nslots) | 1;
        const size_t psm = (size_t)SD_THREADS * pitch * 8;
        const int per_sm = std::max(1, std::min(8, (int)(200 * 1024 / psm)));
        const long long want = ((n + 3) / 4 + SD_THREADS - 1) / SD_THREADS;
        const unsigned pgrid = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() * per_sm));
        // the slot of a * (k - b), when there is exactly one
        int mslot = 0, nmul = 0;
        for (int sl = 1; sl < as.nslots; sl++)
            if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS) {
                mslot = sl;
                nmul++;
            }
        // resident blocks per SM: the shared slices allow per_sm, the
        // registers of the kernel may allow fewer
        auto priv_n = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SD_THREADS, psm) != cudaSuccess || occ < 1)
                occ = 1;
            const unsigned g = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() *
                                                                                   std::min(per_sm, occ)));
            kern<<<g, SD_THREADS, psm, s>>>(ps, ks, as, n, (const long long *)d_nsel, (int)D, pitch, mslot, acc,
                                            d_status);
        };
        auto add_n = [&](auto nsx) { // ADD kernels: MS compile-time
            constexpr int N = decltype(nsx)::value;
            if (mslot == 0 || N < 2)
                priv_n(small_domain_priv_n_kernel<N, true, 0>);
            else if constexpr (N >= 2) {
                if (mslot == 1)
                    priv_n(small_domain_priv_n_kernel<N, true, 1>);
                else if constexpr (N >= 3) {
                    if (mslot == 2)
                        priv_n(small_domain_priv_n_kernel<N, true, 2>);
                    else if constexpr (N >= 4) {
                        if (mslot == 3)
                            priv_n(small_domain_priv_n_kernel<N, true, 3>);
                        else if constexpr (N >= 5)
                            priv_n(small_domain_priv_n_kernel<N, true, 4>);
                    }
                }
            }
        };
        bool add = true; // every slot combines by +
        for (int sl = 1; sl < as.nslots; sl++)
            add = add && as.sop[sl] != TDP_AGG_MIN && as.sop[sl] != TDP_AGG_MAX;
        switch (nmul <= 1 ? as.nslots * 2 + (add ? 1 : 0) : 0) {
        case 2: priv_n(small_domain_priv_n_kernel<1, false, -1>); break;
        case 3: add_n(std::integral_constant<int, 1>()); break;
        case 4: priv_n(small_domain_priv_n_kernel<2, false, -1>); break;
        case 5: add_n(std::integral_constant<int, 2>()); break;
        case 6: priv_n(small_domain_priv_n_kernel<3, false, -1>); break;
        case 7: add_n(std::integral_constant<int, 3>()); break;
        case 8: priv_n(small_domain_priv_n_kernel<4, false, -1>); break;
        case 9: add_n(std::integral_constant<int, 4>()); break;
        case 10: priv_n(small_domain_priv_n_kernel<5, false, -1>); break;
        case 11: add_n(std::integral_constant<int, 5>()); break;
        default:
            cudaFuncSetAttribute(small_domain_priv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
            small_domain_priv_kernel<<<pgrid, SD_THREADS, psm, s>>>(ps, ks, as, n, (const long long *)d_nsel, (int)D,
                                                                    pitch, acc, d_status);
        }
        tdp_status st = launch_status();
        if (st != TDP_OK)
            return st;
        return dense_finalize(ks, as, out, D, acc, capacity, d_ngroups, fin_ws, d_status, s);
    }
    size_t smem = 0;
    int copies = small_domain_copies(D, as.nslots, &smem);
    int blocks_per_sm = copies == 1 ? std::max(1, (int)(200 * 1024 / std::max<size_t>(smem, 1))) : 8;
    blocks_per_sm = std::min(8, blocks_per_sm);
    long long rows = sel ? n : (n + 3) / 4;
    long long want = (rows + SD_THREADS - 1) / SD_THREADS;
    unsigned grid = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() * blocks_per_sm));
    if (sel) {
        cudaFuncSetAttribute(small_domain_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        small_domain_kernel<true><<<grid, SD_THREADS, smem, s>>>(ps, ks, as, n, sel, (const long long *)d_nsel, D,
                                                                copies, acc, d_status);
    } else {
        cudaFuncSetAttribute(small_domain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        small_domain_kernel<false><<<grid, SD_THREADS, smem, s>>>(ps, ks, as, n, nullptr, (const long long *)d_nsel,
                                                                 D, copies, acc, d_status);
    }
    tdp_status st = launch_status();
    if (st != TDP_OK)
        return st;
    return dense_finalize(ks, as, out, D, acc, capacity, d_ngroups, fin_ws, d_status, s);
}

// Partition strategy (groupby_part.cu)
size_t part_ws(long long n, long long D, int nslots);
tdp_status part_run(const PredSet &ps, const KeySet &ks, const AggSet &as, long long D, long long n,
                    const int32_t *sel, const int64_t *d_nsel, const DenseOut &out, long long capacity,
                    int64_t *d_ngroups, void *ws, int32_t *d_status, cudaStream_t s);

// Domain size of bounded key columns (0 when some column has no bounds or
// the product exceeds 2^31).
static long long bounded_domain(const tdp_col *keys, int32_t nkeys)
{
    long long d = 1;
    for (int k = 0; k < nkeys; k++) {
        if (!keys[k].has_bounds || keys[k].hi < keys[k].lo)
            return 0;
        long long sz = keys[k].hi - keys[k].lo + 1;
        if (sz > (1ll << 31) || d * sz > (1ll << 31))
            return 0;
        d *= sz;
    }
    return d;
}

enum GbPath { GB_SMALL, GB_PART, GB_SORT, GB_NONE };

// AUTO: a dense table in shared memory when it fits (small domain), else
// buckets of the dense domain (partition) when the keys are bounded, else
// the sort.
static GbPath choose_path(int32_t strategy, const tdp_col *keys, int32_t nkeys, int nslots)
{
    long long Ds = 0;
    const bool small = keys_small_desc(keys, nkeys, &Ds);
    const long long Db = bounded_domain(keys, nkeys);
    size_t sm = 0;
    switch (strategy) {
    case TDP_GROUPBY_SMALL_DOMAIN: return small ? GB_SMALL : GB_NONE;
    case TDP_GROUPBY_SORT: return GB_SORT;
    case TDP_GROUPBY_PARTITION: return Db > 0 && part_ws(1, Db, nslots) > 0 ? GB_PART : GB_NONE;
    default:
        if (small && small_domain_copies(Ds, nslots, &sm) > 0)
            return GB_SMALL;
        if (Db > 0 && part_ws(1, Db, nslots) > 0)
            return GB_PART;
        return small ? GB_SMALL : GB_SORT;
    }
}

// Sort strategy (groupby_sort.cu)
size_t sort_groupby_ws(long long n, int nkeys, int naggs, int key_bits);
tdp_status sort_groupby_run(const PredSet &ps, const KeySet &ks, int key_bits, const AggSet &as, long long n,
                            const int32_t *sel, const int64_t *d_nsel, const DenseOut &out, long long capacity,
                            int64_t *d_ngroups, void *ws, size_t ws_bytes, int32_t *d_status, cudaStream_t s);
int sort_key_bits(const KeySet &ks);
int sort_key_bits_desc(const tdp_col *keys, int32_t nkeys);

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_groupby_agg_workspace(int64_t n, const tdp_col *keys, int32_t nkeys, int32_t naggs,
                                            int32_t strategy)
{
    if (!keys || nkeys < 1 || nkeys > TDP_MAX_KEYS || naggs < 1 || naggs > TDP_MAX_AGGS)
        return 0;
    // slots: COUNT plus at most one per aggregate
    switch (choose_path(strategy, keys, nkeys, 1 + naggs)) {
    case GB_SMALL: {
        long long D = 0;
        keys_small_desc(keys, nkeys, &D);
        return small_domain_ws(D, naggs);
    }
    case GB_PART: return part_ws(n, bounded_domain(keys, nkeys), 1 + naggs);
    case GB_SORT: {
        int bits = sort_key_bits_desc(keys, nkeys);
        return bits > 0 ? sort_groupby_ws(n, nkeys, naggs, bits) : 0;
    }
    default: return 0;
    }
}

extern "C" tdp_status tdp_groupby_agg(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                                      int64_t n, const int32_t *sel, const int64_t *d_nsel, const int32_t *key_cols,
                                      int32_t nkeys, const tdp_agg *aggs, int32_t naggs, int32_t strategy,
                                      void *const *out_keys, int64_t *const *out_aggs, int64_t capacity,
                                      int64_t *d_ngroups, void *ws, size_t ws_bytes, int32_t *d_status,
                                      tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || !cols || !d_ngroups || capacity < 0 || !out_keys || !out_aggs ||
        (sel && !d_nsel) || strategy < 0 || strategy > 3 || !key_cols || nkeys < 1 || nkeys > TDP_MAX_KEYS)
        return TDP_ERR_INVALID_ARG;
    PredSet ps;
    tdp_status st = make_predset(cols, ncols, preds, npreds, sel ? 0 : n, &ps);
    if (st != TDP_OK)
        return st;
    AggSet as;
    if ((st = make_aggset(cols, ncols, aggs, naggs, sel ? 0 : n, &as)) != TDP_OK)
        return st;
    tdp_col kd[TDP_MAX_KEYS];
    for (int k = 0; k < nkeys; k++) {
        if (key_cols[k] < 0 || key_cols[k] >= ncols)
            return TDP_ERR_INVALID_ARG;
        kd[k] = cols[key_cols[k]];
    }
    // the workspace was sized for 1 + naggs slots; the path is chosen with the
    // same count so that both agree
    const GbPath path = choose_path(strategy, kd, nkeys, 1 + naggs);
    if (path == GB_NONE)
        return TDP_ERR_INVALID_ARG;
    // the group count is this call's output whatever path runs (0 if no row qualifies)
    if (cudaMemsetAsync(d_ngroups, 0, sizeof(int64_t), (cudaStream_t)stream) != cudaSuccess)
        return TDP_ERR_CUDA;
    KeySet ks;
    long long D = 0;
    if ((st = make_keyset(cols, ncols, key_cols, nkeys, sel ? 0 : n, &ks, path != GB_SORT, &D)) != TDP_OK)
        return st;
    DenseOut out;
    for (int k = 0; k < TDP_MAX_KEYS; k++) {
        out.key_out[k] = k < nkeys ? out_keys[k] : nullptr;
        out.key_dt[k] = k < nkeys ? cols[key_cols[k]].dtype : 0;
        if (k < nkeys && capacity > 0 && !out.key_out[k])
            return TDP_ERR_INVALID_ARG;
    }
    for (int a = 0; a < TDP_MAX_AGGS; a++) {
        out.agg_out[a] = a < naggs ? (long long *)out_aggs[a] : nullptr;
        if (a < naggs && capacity > 0 && !out.agg_out[a])
            return TDP_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (path == GB_SMALL) {
        if (!ws || ws_bytes < small_domain_ws(D, naggs))
            return TDP_ERR_WORKSPACE_TOO_SMALL;
        return small_domain_run(ps, ks, as, D, n, sel, d_nsel, out, capacity, d_ngroups, ws, d_status, s);
    }
    if (path == GB_PART) {
        if (!ws || ws_bytes < part_ws(n, D, 1 + naggs))
            return TDP_ERR_WORKSPACE_TOO_SMALL;
        return part_run(ps, ks, as, D, n, sel, d_nsel, out, capacity, d_ngroups, ws, d_status, s);
    }
    int bits = sort_key_bits(ks);
    if (bits <= 0)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (!ws || ws_bytes < sort_groupby_ws(n, nkeys, naggs, bits))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    return sort_groupby_run(ps, ks, bits, as, n, sel, d_nsel, out, capacity, d_ngroups, ws, ws_bytes, d_status, s);
}
