// K6/K7: open-addressing hash equi-join (build, probe, fused probe+group-by).
//
// Table: nslots (power of two) 64-bit slots in HBM, slot = (uint32(key) << 32)
// | payload, empty = all ones (so the pair key = -1, payload = -1 cannot be
// stored; the build flags it as TDP_ERR_OVERFLOW).  Multiplicative (Fibonacci)
// hash, linear probing, one 64-bit CAS per insert, probe length bounded by
// min(nslots, 65536).
//
// Probe: same tile structure as the filter (256 threads x 16 rows, 4 steps of
// 128 rows per warp, lane = 4 consecutive rows): the probe-side predicates
// and keys are read with 16-byte loads, the 16 lookups of a thread advance
// through their collision chains in lock-step rounds (each round issues all
// outstanding slot loads before examining any, so a thread waits for its
// longest chain rather than the sum of its chains), and matches are compacted
// with ballots + decoupled look-back so that the output keeps probe order.
//
// Probe + aggregate: the build payload is the group key (dense range
// [lo, hi]); matched rows are added into a per-block shared-memory cache of
// 2048 groups (open addressing on the group id), which absorbs Zipf-hot
// groups; groups that find no cache slot go straight to the global dense
// accumulator table with 64-bit atomics.  Cache contents are merged into the
// global table at the end, then the non-empty groups are compacted in order.
#include "filter_api.cuh"
#include "groupby.cuh"

namespace tdp {

constexpr unsigned long long EMPTY_SLOT = ~0ull;
// Longest probe sequence walked by a build insert or a lookup.  Linear probing
// at load <= 1/2 needs a handful of steps; a longer run means a (nearly) full
// table, which is reported as TDP_ERR_CAPACITY instead of being walked.
constexpr unsigned long long MAX_PROBE = 1ull << 16;

__device__ __forceinline__ unsigned hash_slot(int key, int lg)
{
    return ((unsigned)key * 0x9E3779B1u) >> (32 - lg);
}

__global__ void fill_empty_kernel(unsigned long long *table, long long nslots)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < nslots; i += (long long)gridDim.x * blockDim.x)
        table[i] = EMPTY_SLOT;
}

__global__ void join_build_kernel(PredSet ps, const int32_t *__restrict__ key, const int32_t *__restrict__ payload,
                                  long long n, const long long *d_n, unsigned long long *table, int lg,
                                  int32_t *d_status)
{
    if (d_n)
        n = min(*d_n, n);
    const unsigned long long mask = (1ull << lg) - 1;
    const unsigned long long steps = mask + 1 < MAX_PROBE ? mask + 1 : MAX_PROBE;
    int err = 0;
    // 4 consecutive rows per thread: predicate, key and payload columns are
    // read with vector loads before any insert starts
    const long long r0 = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r0 >= n)
        return;
    unsigned m = eval_preds4(ps, r0, n);
    if (!m)
        return;
    int k[4];
    unsigned p[4];
    const bool full = r0 + 3 < n && ((uintptr_t)key % 16) == 0 && (!payload || ((uintptr_t)payload % 16) == 0);
    if (full) {
        int4 kk = __ldg((const int4 *)(key + r0));
        k[0] = kk.x, k[1] = kk.y, k[2] = kk.z, k[3] = kk.w;
        if (payload) {
            int4 pp = __ldg((const int4 *)(payload + r0));
            p[0] = pp.x, p[1] = pp.y, p[2] = pp.z, p[3] = pp.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            k[e] = (m >> e & 1) ? key[r0 + e] : 0;
            p[e] = (m >> e & 1) && payload ? (unsigned)payload[r0 + e] : 0u;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
        if (!(m >> e & 1))
            continue;
        unsigned pe = payload ? p[e] : (unsigned)(r0 + e);
        unsigned long long v = ((unsigned long long)(unsigned)k[e] << 32) | pe;
        if (v == EMPTY_SLOT) {
            err |= TDP_ERR_OVERFLOW;
            continue;
        }
        unsigned long long h = hash_slot(k[e], lg);
        bool done = false;
        for (unsigned long long probe = 0; probe < steps; probe++) {
            unsigned long long prev = atomicCAS(&table[h], EMPTY_SLOT, v);
            if (prev == EMPTY_SLOT) {
                done = true;
                break;
            }
            if ((unsigned)(prev >> 32) == (unsigned)k[e]) {
                err |= TDP_ERR_DUP_BUILD_KEY;
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done)
            err |= TDP_ERR_CAPACITY;
    }
    if (err)
        set_status(d_status, err);
}

constexpr int JP_THREADS = 256;
constexpr int JP_STEPS = 2;
constexpr int JP_WARP_ROWS = JP_STEPS * 128;
constexpr int JP_TILE = JP_THREADS / 32 * JP_WARP_ROWS;
constexpr int JP_ROWS = JP_STEPS * 4; // rows per thread

// Reads the probe keys of the 16 rows of a thread and resolves them.  idx0:
// the thread's first index (multiple of 4); row r = j*4 + e is idx0 + j*128 + e
// (or sel[...] of it).  All unresolved lookups advance together: every round
// issues the next slot load of each of them before any is examined, so a
// thread waits for its longest collision chain, not for the sum of its chains.
// On return bit r of `hit` is set for rows that qualify and match; pay[r] is
// the payload, key[r] the probe key, row[r] the row id.
__device__ __forceinline__ unsigned probe16(const unsigned long long *table, int lg, const PredSet &ps,
                                            const int32_t *keycol, bool key_vec, const int32_t *sel, long long m,
                                            long long idx0, unsigned (&pay)[JP_ROWS], int (&key)[JP_ROWS],
                                            int (&row)[JP_ROWS], bool &gave_up)
{
    unsigned hit = 0;
#pragma unroll
    for (int j = 0; j < JP_STEPS; j++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            long long i = idx0 + j * 128 + e;
            row[j * 4 + e] = i < m ? (sel ? sel[i] : (int)i) : -1;
            hit |= (i < m) ? (1u << (j * 4 + e)) : 0u;
        }
    if (ps.n > 0) {
        if (!sel) {
            for (int p = 0; p < ps.n; p++) {
                long long v[JP_STEPS][4];
                load_rows<JP_STEPS>(ps.col[p], ps.dt[p], ps.vec_ok[p], idx0, m, v);
#pragma unroll
                for (int j = 0; j < JP_STEPS; j++)
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        if (!cmp_holds(v[j][e], ps.cmp[p], ps.lit[p]))
                            hit &= ~(1u << (j * 4 + e));
            }
        } else {
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                if ((hit >> r & 1) && !eval_preds1(ps, row[r]))
                    hit &= ~(1u << r);
        }
    }
    if (!sel && key_vec && idx0 + (JP_STEPS - 1) * 128 + 3 < m) {
        int4 w[JP_STEPS];
#pragma unroll
        for (int j = 0; j < JP_STEPS; j++)
            w[j] = __ldg((const int4 *)(keycol + idx0 + j * 128));
#pragma unroll
        for (int j = 0; j < JP_STEPS; j++)
            key[j * 4 + 0] = w[j].x, key[j * 4 + 1] = w[j].y, key[j * 4 + 2] = w[j].z, key[j * 4 + 3] = w[j].w;
    } else {
#pragma unroll
        for (int r = 0; r < JP_ROWS; r++)
            key[r] = (hit >> r & 1) ? keycol[row[r]] : 0;
    }
    const unsigned mask = (unsigned)((1ull << lg) - 1);
    const unsigned long long steps = (unsigned long long)mask + 1 < MAX_PROBE ? (unsigned long long)mask + 1 : MAX_PROBE;
    unsigned long long s[JP_ROWS];
    unsigned h[JP_ROWS];
    unsigned act = hit;
#pragma unroll
    for (int r = 0; r < JP_ROWS; r++) {
        h[r] = hash_slot(key[r], lg);
        s[r] = (act >> r & 1) ? __ldg(table + h[r]) : EMPTY_SLOT;
    }
    for (unsigned long long round = 0; act && round < steps; round++) {
#pragma unroll
        for (int r = 0; r < JP_ROWS; r++) {
            if (!(act >> r & 1))
                continue;
            if (s[r] == EMPTY_SLOT) {
                act &= ~(1u << r);
                hit &= ~(1u << r);
            } else if ((unsigned)(s[r] >> 32) == (unsigned)key[r]) {
                act &= ~(1u << r);
                pay[r] = (unsigned)s[r];
            } else {
                h[r] = (h[r] + 1) & mask;
            }
        }
#pragma unroll
        for (int r = 0; r < JP_ROWS; r++)
            if (act >> r & 1)
                s[r] = __ldg(table + h[r]);
    }
    if (act) { // a chain longer than MAX_PROBE: reported, rows dropped
        gave_up = true;
        hit &= ~act;
    }
    return hit;
}

__global__ void __launch_bounds__(JP_THREADS) join_probe_kernel(const unsigned long long *__restrict__ table, int lg,
                                                                PredSet ps, const int32_t *__restrict__ key,
                                                                bool key_vec, long long n, const int32_t *sel,
                                                                const long long *d_nsel, int32_t *out_row,
                                                                int32_t *out_payload, GatherSet gs, long long cap,
                                                                long long *d_count, unsigned long long *tile_status,
                                                                unsigned *ticket, int32_t *d_status, uint32_t limit,
                                                                long long num_tiles)
{
    __shared__ long long s_tile;
    __shared__ unsigned s_warp_tot[JP_THREADS / 32];
    __shared__ unsigned s_warp_excl[JP_THREADS / 32];
    __shared__ unsigned long long s_excl;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long m = d_nsel ? min(*d_nsel, n) : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long idx0 = tile * JP_TILE + (long long)warp * JP_WARP_ROWS + 4 * lane;

    unsigned pay[JP_ROWS];
    int keys[JP_ROWS], rows[JP_ROWS];
    bool gave_up = false;
    const unsigned hit = probe16(table, lg, ps, key, key_vec, sel, m, idx0, pay, keys, rows, gave_up);
    if (gave_up)
        set_status(d_status, TDP_ERR_CAPACITY);

    const unsigned lt = lanemask_lt();
    unsigned step_cnt[JP_STEPS], lane_pref[JP_STEPS], warp_tot = 0;
#pragma unroll
    for (int j = 0; j < JP_STEPS; j++) {
        unsigned c = 0, pre = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            unsigned b = __ballot_sync(0xffffffffu, (hit >> (j * 4 + e)) & 1u);
            c += __popc(b);
            pre += __popc(b & lt);
        }
        step_cnt[j] = c;
        lane_pref[j] = pre;
        warp_tot += c;
    }
    if (lane == 0)
        s_warp_tot[warp] = warp_tot;
    __syncthreads();
    if (warp == 0) {
        unsigned t = lane < JP_THREADS / 32 ? s_warp_tot[lane] : 0, incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += u;
        }
        if (lane < JP_THREADS / 32)
            s_warp_excl[lane] = incl - t;
        unsigned long long agg = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long excl = lookback_exclusive(tile_status, tile, agg, limit, d_status);
        if (lane == 0) {
            s_excl = excl;
            if (tile == num_tiles - 1) {
                long long total = (long long)(excl + agg);
                *d_count = total;
                if (total > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    // output slot of every hit (rows of a step land at consecutive slots)
    long long outp[JP_ROWS];
    {
        long long pos = (long long)s_excl + s_warp_excl[warp];
#pragma unroll
        for (int j = 0; j < JP_STEPS; j++) {
            long long p = pos + lane_pref[j];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                outp[j * 4 + e] = p;
                p += (hit >> (j * 4 + e)) & 1;
            }
            pos += step_cnt[j];
        }
    }
    const unsigned wr = hit; // rows written (subject to capacity)
#pragma unroll
    for (int r = 0; r < JP_ROWS; r++) {
        if (!(wr >> r & 1) || outp[r] >= cap)
            continue;
        if (out_row)
            out_row[outp[r]] = rows[r];
        if (out_payload)
            out_payload[outp[r]] = (int32_t)pay[r];
    }
    // gathers: all loads of a column are issued before its stores
    for (int g = 0; g < gs.n; g++) {
        const void *col = gs.col[g];
        void *out = gs.out[g];
        if (col == (const void *)key) { // the probe key is already in a register
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                if ((wr >> r & 1) && outp[r] < cap)
                    ((int *)out)[outp[r]] = keys[r];
            continue;
        }
        if (gs.size[g] == 8) {
            long long v[JP_ROWS];
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                v[r] = (wr >> r & 1) ? __ldg((const long long *)col + rows[r]) : 0;
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                if ((wr >> r & 1) && outp[r] < cap)
                    ((long long *)out)[outp[r]] = v[r];
        } else if (gs.size[g] == 4) {
            int v[JP_ROWS];
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                v[r] = (wr >> r & 1) ? __ldg((const int *)col + rows[r]) : 0;
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++)
                if ((wr >> r & 1) && outp[r] < cap)
                    ((int *)out)[outp[r]] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < JP_ROWS; r++) {
                if (!(wr >> r & 1) || outp[r] >= cap)
                    continue;
                if (gs.size[g] == 2)
                    ((uint16_t *)out)[outp[r]] = ((const uint16_t *)col)[rows[r]];
                else
                    ((uint8_t *)out)[outp[r]] = ((const uint8_t *)col)[rows[r]];
            }
        }
    }
}

// ------------------------------------------------------- probe + aggregate

constexpr int GJ_CACHE = 2048;
constexpr int GJ_PROBES = 8;

__global__ void __launch_bounds__(JP_THREADS) join_probe_agg_kernel(const unsigned long long *__restrict__ table,
                                                                    int lg, PredSet ps,
                                                                    const int32_t *__restrict__ key, bool key_vec,
                                                                    long long n, const long long *d_n,
                                                                    long long lo, long long D, AggSet as,
                                                                    long long *gacc, int32_t *d_status)
{
    if (d_n)
        n = min(*d_n, n);
    extern __shared__ long long gj_smem[];
    const int NS = as.nslots;
    long long *s_acc = gj_smem;                               // [GJ_CACHE][NS]
    unsigned *s_key = (unsigned *)(gj_smem + GJ_CACHE * NS);  // [GJ_CACHE], gid + 1, 0 = empty
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    if (threadIdx.x <= TDP_MAX_AGGS) {
        int s = threadIdx.x, op = TDP_AGG_SUM;
        for (int a = 0; a < as.n; a++)
            if (as.slot[a] == s && s != 0)
                op = as.op[a];
        s_ops[s] = op;
        s_init[s] = slot_init(as, s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < GJ_CACHE; e += JP_THREADS) {
        s_key[e] = 0;
        for (int s = 0; s < NS; s++)
            s_acc[e * NS + s] = s_init[s];
    }
    __syncthreads();
    bool bad = false;
    const long long stride = (long long)gridDim.x * JP_TILE;
    for (long long base = (long long)blockIdx.x * JP_TILE; base < n; base += stride) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const long long idx0 = base + (long long)warp * JP_WARP_ROWS + 4 * lane;
        unsigned pay[JP_ROWS];
        int keys[JP_ROWS], rows[JP_ROWS];
        bool gave_up = false;
        const unsigned hit = probe16(table, lg, ps, key, key_vec, nullptr, n, idx0, pay, keys, rows, gave_up);
        if (gave_up)
            set_status(d_status, TDP_ERR_CAPACITY);
#pragma unroll
        for (int j = 0; j < JP_STEPS; j++) {
            unsigned hj = (hit >> (4 * j)) & 0xfu;
            if (!hj)
                continue;
            long long *dst[4] = {nullptr, nullptr, nullptr, nullptr};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (!(hj >> e & 1))
                    continue;
                long long gid = (long long)(int)pay[j * 4 + e] - lo;
                if (gid < 0 || gid >= D) {
                    bad = true;
                    hj &= ~(1u << e);
                    continue;
                }
                // find / claim a cache slot
                unsigned tag = (unsigned)gid + 1u;
                unsigned h = ((unsigned)gid * 0x9E3779B1u) >> 21; // 11 bits: GJ_CACHE = 2048
                long long *d = nullptr;
                for (int q = 0; q < GJ_PROBES; q++) {
                    unsigned cur = s_key[h];
                    if (cur == 0)
                        cur = atomicCAS(&s_key[h], 0u, tag);
                    if (cur == 0 || cur == tag) {
                        d = s_acc + h * NS;
                        break;
                    }
                    h = (h + 1) & (GJ_CACHE - 1);
                }
                if (!d)
                    d = gacc + gid * NS;
                dst[e] = d;
                atomicAdd((unsigned long long *)&d[0], 1ull);
            }
            if (!hj)
                continue;
            for (int a = 0; a < as.n; a++) {
                if (as.op[a] == TDP_AGG_COUNT)
                    continue;
                long long x[4], y[4] = {0, 0, 0, 0};
                load4_int(as.a[a], as.adt[a], as.avec[a], idx0 + j * 128, n, x);
                if (as.op[a] == TDP_AGG_SUM_MUL_KMINUS)
                    load4_int(as.b[a], as.bdt[a], as.bvec[a], idx0 + j * 128, n, y);
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (hj >> e & 1)
                        acc_update(&dst[e][as.slot[a]], as.op[a], agg_value(as, a, x[e], y[e]));
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    __syncthreads();
    for (int e = threadIdx.x; e < GJ_CACHE; e += JP_THREADS) {
        unsigned tag = s_key[e];
        if (!tag)
            continue;
        long long gid = (long long)tag - 1;
        for (int s = 0; s < NS; s++) {
            long long v = s_acc[e * NS + s];
            if (v != s_init[s])
                acc_update(&gacc[gid * NS + s], s_ops[s], v);
        }
    }
}

static int log2_slots(long long nslots)
{
    int lg = 0;
    while ((1ll << lg) < nslots)
        lg++;
    return lg;
}

static bool pow2_ok(long long nslots) { return nslots >= 2 && nslots <= (1ll << 32) && (nslots & (nslots - 1)) == 0; }

} // namespace tdp

using namespace tdp;

extern "C" int64_t tdp_join_default_slots(int64_t n_keys)
{
    long long s = 2;
    while (s < 2 * n_keys)
        s <<= 1;
    return s;
}

extern "C" tdp_status tdp_join_build(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                                     int64_t n, const int64_t *d_n, int32_t key_col, int32_t payload_col, uint32_t flags,
                                     uint64_t *table, int64_t nslots, int32_t *d_status, tdp_stream_t stream)
{
    (void)flags;
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !pow2_ok(nslots) || key_col < 0 || key_col >= ncols ||
        payload_col >= ncols)
        return TDP_ERR_INVALID_ARG;
    if (cols[key_col].dtype != TDP_I32 || (payload_col >= 0 && cols[payload_col].dtype != TDP_I32))
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (cols[key_col].n < n || (payload_col >= 0 && cols[payload_col].n < n))
        return TDP_ERR_INVALID_ARG;
    PredSet ps;
    tdp_status st = make_predset(cols, ncols, preds, npreds, n, &ps);
    if (st != TDP_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    fill_empty_kernel<<<(unsigned)std::min<long long>((nslots + 255) / 256, (long long)num_sms() * 8), 256, 0, s>>>(
        (unsigned long long *)table, nslots);
    if (n > 0) {
        // one thread per 4 rows (the kernel is not grid-strided)
        unsigned grid = (unsigned)((n + 1023) / 1024);
        join_build_kernel<<<grid, 256, 0, s>>>(ps, (const int32_t *)cols[key_col].data,
                                               payload_col >= 0 ? (const int32_t *)cols[payload_col].data : nullptr,
                                               n, (const long long *)d_n, (unsigned long long *)table,
                                               log2_slots(nslots), d_status);
    }
    return launch_status();
}

extern "C" size_t tdp_join_probe_workspace(int64_t n)
{
    long long tiles = (n + JP_TILE - 1) / JP_TILE;
    return align_up(16 + (size_t)tiles * 8, 256);
}

extern "C" tdp_status tdp_join_probe(const uint64_t *table, int64_t nslots, const tdp_col *cols, int32_t ncols,
                                     const tdp_pred *preds, int32_t npreds, int64_t n, const int32_t *sel,
                                     const int64_t *d_nsel, int32_t key_col, int32_t *out_probe_row,
                                     int32_t *out_payload, const int32_t *gather_cols, int32_t ngather,
                                     void *const *gather_out, int64_t capacity, int64_t *d_count, void *ws,
                                     size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !pow2_ok(nslots) || key_col < 0 || key_col >= ncols ||
        !d_count || capacity < 0 || (sel && !d_nsel))
        return TDP_ERR_INVALID_ARG;
    if (cols[key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    const long long rows_req = sel ? 0 : n;
    if (cols[key_col].n < rows_req)
        return TDP_ERR_INVALID_ARG;
    PredSet ps;
    tdp_status st = make_predset(cols, ncols, preds, npreds, rows_req, &ps);
    if (st != TDP_OK)
        return st;
    GatherSet gs;
    if ((st = make_gatherset(cols, ncols, gather_cols, ngather, gather_out, rows_req, &gs)) != TDP_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, 8, s);
        return launch_status();
    }
    if (!ws || ws_bytes < tdp_join_probe_workspace(n))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    long long tiles = (n + JP_TILE - 1) / JP_TILE;
    cudaMemsetAsync(ws, 0, 16 + (size_t)tiles * 8, s);
    const int32_t *key = (const int32_t *)cols[key_col].data;
    join_probe_kernel<<<(unsigned)tiles, JP_THREADS, 0, s>>>(
        (const unsigned long long *)table, log2_slots(nslots), ps, key, ((uintptr_t)key % 16) == 0, n, sel,
        (const long long *)d_nsel, out_probe_row, out_payload, gs, capacity, (long long *)d_count,
        (unsigned long long *)((char *)ws + 16), (unsigned *)ws, d_status, spin_limit(), tiles);
    return launch_status();
}

extern "C" size_t tdp_join_workspace(int64_t n_build, int64_t n_probe, int64_t nslots)
{
    if (nslots <= 0)
        nslots = tdp_join_default_slots(n_build);
    return align_up((size_t)nslots * 8, 256) + tdp_join_probe_workspace(n_probe);
}

extern "C" tdp_status tdp_join(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                               int32_t nbuild_preds, int64_t n_build, int32_t build_key_col, int32_t build_payload_col,
                               const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                               int32_t nprobe_preds, int64_t n_probe, int32_t probe_key_col, int64_t nslots,
                               int32_t *out_probe_row, int32_t *out_payload, const int32_t *gather_cols,
                               int32_t ngather, void *const *gather_out, int64_t capacity, int64_t *d_count,
                               void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (nslots <= 0)
        nslots = tdp_join_default_slots(n_build);
    if (!ws || ws_bytes < tdp_join_workspace(n_build, n_probe, nslots))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    uint64_t *table = (uint64_t *)ws;
    char *pws = (char *)ws + align_up((size_t)nslots * 8, 256);
    tdp_status st = tdp_join_build(build_cols, nbuild_cols, build_preds, nbuild_preds, n_build, nullptr, build_key_col,
                                   build_payload_col, TDP_JOIN_UNIQUE_BUILD, table, nslots, d_status, stream);
    if (st != TDP_OK)
        return st;
    return tdp_join_probe(table, nslots, probe_cols, nprobe_cols, probe_preds, nprobe_preds, n_probe, nullptr,
                          nullptr, probe_key_col, out_probe_row, out_payload, gather_cols, ngather, gather_out,
                          capacity, d_count, pws, tdp_join_probe_workspace(n_probe), d_status, stream);
}

extern "C" size_t tdp_join_probe_agg_workspace(int64_t n, int64_t domain, int32_t naggs)
{
    (void)n;
    if (domain <= 0)
        return 0;
    return align_up((size_t)domain * (1 + naggs) * 8, 256) + dense_finalize_ws(domain);
}

extern "C" tdp_status tdp_join_probe_agg(const uint64_t *table, int64_t nslots, const tdp_col *cols, int32_t ncols,
                                         const tdp_pred *preds, int32_t npreds, int64_t n, const int64_t *d_n,
                                         int32_t key_col, int64_t payload_lo, int64_t payload_hi, const tdp_agg *aggs, int32_t naggs,
                                         int32_t *out_keys, int64_t *const *out_aggs, int64_t capacity,
                                         int64_t *d_ngroups, void *ws, size_t ws_bytes, int32_t *d_status,
                                         tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !pow2_ok(nslots) || key_col < 0 || key_col >= ncols ||
        !d_ngroups || capacity < 0 || payload_hi < payload_lo || payload_hi - payload_lo >= (1ll << 31) ||
        !out_aggs || (capacity > 0 && !out_keys))
        return TDP_ERR_INVALID_ARG;
    if (cols[key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (cols[key_col].n < n)
        return TDP_ERR_INVALID_ARG;
    PredSet ps;
    tdp_status st = make_predset(cols, ncols, preds, npreds, n, &ps);
    if (st != TDP_OK)
        return st;
    AggSet as;
    if ((st = make_aggset(cols, ncols, aggs, naggs, n, &as)) != TDP_OK)
        return st;
    const long long D = payload_hi - payload_lo + 1;
    if (!ws || ws_bytes < tdp_join_probe_agg_workspace(n, D, naggs))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    long long *acc = (long long *)ws;
    void *fin_ws = (char *)ws + align_up((size_t)D * as.nslots * 8, 256);
    dense_acc_init_kernel<<<(unsigned)std::min<long long>((D * as.nslots + 255) / 256, 4096), 256, 0, s>>>(as, D,
                                                                                                         acc);
    if (n > 0) {
        const size_t smem = (size_t)GJ_CACHE * as.nslots * 8 + GJ_CACHE * 4;
        if (cudaFuncSetAttribute(join_probe_agg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return TDP_ERR_CUDA;
        int per_sm = std::max(1, std::min(4, (int)((200 * 1024) / smem)));
        long long want = (n + JP_TILE - 1) / JP_TILE;
        unsigned grid = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() * per_sm));
        const int32_t *key = (const int32_t *)cols[key_col].data;
        join_probe_agg_kernel<<<grid, JP_THREADS, smem, s>>>((const unsigned long long *)table, log2_slots(nslots), ps,
                                                            key, ((uintptr_t)key % 16) == 0, n,
                                                            (const long long *)d_n, payload_lo, D, as, acc, d_status);
    }
    if ((st = launch_status()) != TDP_OK)
        return st;
    KeySet ks;
    ks.n = 1;
    for (int k = 0; k < TDP_MAX_KEYS; k++) {
        ks.col[k] = nullptr;
        ks.dt[k] = TDP_I32;
        ks.vec_ok[k] = 0;
        ks.lo[k] = k == 0 ? payload_lo : 0;
        ks.size[k] = k == 0 ? D : 0;
        ks.stride[k] = k == 0 ? 1 : 0;
    }
    DenseOut out;
    for (int k = 0; k < TDP_MAX_KEYS; k++) {
        out.key_out[k] = k == 0 ? (void *)out_keys : nullptr;
        out.key_dt[k] = TDP_I32;
    }
    for (int a = 0; a < TDP_MAX_AGGS; a++)
        out.agg_out[a] = a < naggs ? (long long *)out_aggs[a] : nullptr;
    return dense_finalize(ks, as, out, D, acc, capacity, d_ngroups, fin_ws, d_status, s);
}
