// K4/K5 for a bounded key domain too large for one shared-memory table
// (strategy TDP_GROUPBY_PARTITION): the sort of Sec. 4's sort-based group-by
// taken only as far as the aggregation needs it.
//
// The key tuple maps to a dense group id gid in [0, D) (as in the small-domain
// strategy).  Buckets of B consecutive gids (B = 4096 when one sum is
// carried) are small enough for a dense accumulator table in shared memory:
//   1. count:    rows per bucket (shared-memory histograms, one global add per
//                non-empty bucket per block);
//   2. scan:     bucket start offsets (one block);
//   3. scatter:  every row's gid and slot values (the aggregate inputs,
//                a*(k-b) already formed) go to its bucket's segment; each
//                warp reserves room for the rows it sends to one bucket with
//                one atomic on the bucket's cursor (rows of a bucket are not
//                kept in input order: the aggregates are exact integer sums,
//                minima and maxima, so their order does not matter);
//   4. reduce:   one block per bucket (block index = bucket index) adds its
//                segment into a B x nslots table in shared memory, ranks the
//                non-empty gids with ballots, takes its output offset from a
//                decoupled look-back over the buckets before it, and writes
//                its groups in ascending gid order, which is ascending key
//                order.
// Traffic per row: keys and aggregate inputs read twice (count, scatter),
// 4 + 8 x (nslots - 1) bytes written and read back once.
#include <algorithm>

#include "groupby.cuh"

namespace tdp {

constexpr int GP_THREADS = 512;  // reduce pass
constexpr int GS_THREADS = 1024; // count and scatter passes (rows in flight per SM)
constexpr int GP_MAX_BUCKETS = 16384;
constexpr size_t GP_TABLE_BYTES = 64 * 1024; // dense table of one bucket

struct PartPlan {
    int bw;       // log2(B)
    long long nb; // buckets
};

// Bucket width: the largest B <= 4096 whose B x nslots x 8 bytes fit the table
// budget.  False when the domain needs more than GP_MAX_BUCKETS buckets.
bool part_plan(long long D, int nslots, PartPlan *pp)
{
    int bw = 12;
    while (bw > 5 && ((size_t)1 << bw) * nslots * 8 > GP_TABLE_BYTES)
        bw--;
    const long long nb = (D + (1ll << bw) - 1) >> bw;
    if (D < 1 || D > (1ll << 31) || nb > GP_MAX_BUCKETS)
        return false;
    pp->bw = bw;
    pp->nb = nb;
    return true;
}

// The rows of block g: a contiguous chunk of the dense rows (or of the row
// list), the same chunk in the count and the scatter pass (both run on the
// same grid and read the same device row count).
template <bool SEL>
__device__ __forceinline__ void block_chunk(long long n, const long long *d_nsel, long long &c0, long long &c1)
{
    const long long total = SEL ? min(*d_nsel, n) : (d_nsel ? min(*d_nsel, n) : n);
    const long long unit = SEL ? GS_THREADS : 4 * GS_THREADS;
    long long chunk = (total + gridDim.x - 1) / gridDim.x;
    chunk = (chunk + unit - 1) / unit * unit;
    c0 = min(total, (long long)blockIdx.x * chunk);
    c1 = min(total, c0 + chunk);
}

// Rows of the block's chunk, with the predicates and the key bounds applied:
// a dense scan takes 4 rows a thread and step (vector loads), a row list one
// entry.  Calls f(row, gid) for every row position, gid = -1 for rows that
// do not qualify or lie past the chunk; every lane of a warp makes the same
// number of calls (f may be warp-wide).  Returns false when some key was out
// of bounds.
template <bool SEL, class F>
__device__ __forceinline__ bool for_rows(const PredSet &ps, const KeySet &ks, long long n, const int32_t *sel,
                                         const long long *d_nsel, F f)
{
    long long c0, c1;
    block_chunk<SEL>(n, d_nsel, c0, c1);
    bool bad = false;
    if (!SEL) {
        const long long off = (long long)(threadIdx.x & ~31) * 4 + (threadIdx.x & 31) * 4;
        for (long long sb = c0; sb < c1; sb += 4 * GS_THREADS) {
            const long long r = sb + off;
            unsigned m = eval_preds4(ps, r, c1);
            long long gid[4] = {0, 0, 0, 0};
            for (int k = 0; k < ks.n; k++) {
                long long v[4];
                load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, c1, v);
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
                f(r + j, (m >> j & 1) ? gid[j] : -1ll);
        }
    } else {
        for (long long sb = c0; sb < c1; sb += GS_THREADS) {
            const long long i = sb + threadIdx.x;
            long long gid = -1;
            long long row = 0;
            if (i < c1) {
                row = sel[i];
                if (eval_preds1(ps, row)) {
                    if (!row_gid(ks, row, gid)) {
                        gid = -1;
                        bad = true;
                    }
                }
            }
            f(row, gid);
        }
    }
    return !bad;
}

// Count: the block's rows per bucket (shared-memory histogram), then one add
// per non-empty bucket to the bucket's total; the value the add returns is
// this block's offset within the bucket, kept in boff[block][bucket] for the
// scatter pass.
template <bool SEL>
__global__ void __launch_bounds__(GS_THREADS) part_count_kernel(PredSet ps, KeySet ks, long long n,
                                                                const int32_t *sel, const long long *d_nsel,
                                                                int bw, int nb, unsigned *hist, unsigned *boff,
                                                                int32_t *d_status)
{
    extern __shared__ unsigned gp_hist[];
    for (int i = threadIdx.x; i < nb; i += GS_THREADS)
        gp_hist[i] = 0;
    __syncthreads();
    const bool ok = for_rows<SEL>(ps, ks, n, sel, d_nsel, [&](long long, long long gid) {
        if (gid >= 0)
            atomicAdd(&gp_hist[gid >> bw], 1u);
    });
    if (!ok)
        set_status(d_status, TDP_ERR_OVERFLOW);
    __syncthreads();
    unsigned *my = boff + (size_t)blockIdx.x * nb;
    for (int i = threadIdx.x; i < nb; i += GS_THREADS) {
        const unsigned c = gp_hist[i];
        my[i] = c ? atomicAdd(&hist[i], c) : 0u;
    }
}

// Exclusive scan of hist[nb] into start[0..nb] (one block of 1024 threads,
// 16 buckets a thread).
__global__ void __launch_bounds__(1024) part_scan_kernel(const unsigned *hist, int nb, unsigned *start)
{
    __shared__ unsigned s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned v[16], sum = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int b = tid * 16 + i;
        v[i] = b < nb ? hist[b] : 0u;
        sum += v[i];
    }
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    unsigned wpre = 0, total = 0;
    for (int w = 0; w < 32; w++) {
        const unsigned t = s_warp[w];
        wpre += w < warp ? t : 0;
        total += t;
    }
    unsigned run = wpre + incl - sum;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const int b = tid * 16 + i;
        if (b < nb)
            start[b] = run;
        run += v[i];
    }
    if (tid == 0)
        start[nb] = total;
}

// Scatter: the rows of the block's chunk to their buckets' segments with
// (gid, slot values), at start[bucket] + the block's offset within the bucket
// + a shared-memory counter (no global atomics).
template <bool SEL>
__global__ void __launch_bounds__(GS_THREADS) part_scatter_kernel(PredSet ps, KeySet ks, AggSet as, long long n,
                                                                  const int32_t *sel, const long long *d_nsel,
                                                                  int bw, int nb, const unsigned *start,
                                                                  const unsigned *boff, uint32_t *out_gid,
                                                                  long long *out_val, long long val_stride)
{
    extern __shared__ unsigned gp_base[];
    const unsigned *my = boff + (size_t)blockIdx.x * nb;
    for (int i = threadIdx.x; i < nb; i += GS_THREADS)
        gp_base[i] = start[i] + my[i];
    __syncthreads();
    const int NS = as.nslots;
    if (SEL) {
        for_rows<SEL>(ps, ks, n, sel, d_nsel, [&](long long row, long long gid) {
            if (gid < 0)
                return;
            const unsigned pos = atomicAdd(&gp_base[gid >> bw], 1u);
            out_gid[pos] = (uint32_t)gid;
            for (int s = 1; s < NS; s++)
                out_val[(s - 1) * val_stride + pos] = slot_value(as, s, row);
        });
        return;
    }
    long long c0, c1;
    block_chunk<false>(n, d_nsel, c0, c1);
    const long long off = (long long)threadIdx.x * 4;
    for (long long sb = c0; sb < c1; sb += 4 * GS_THREADS) {
        const long long r = sb + off;
        unsigned m = eval_preds4(ps, r, c1);
        long long gid[4] = {0, 0, 0, 0};
        for (int k = 0; k < ks.n; k++) {
            long long v[4];
            load4_int(ks.col[k], ks.dt[k], ks.vec_ok[k], r, c1, v);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const long long d = v[j] - ks.lo[k];
                if (d < 0 || d >= ks.size[k])
                    m &= ~(1u << j); // flagged by the count pass
                gid[j] += d * ks.stride[k];
            }
        }
        unsigned pos[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            pos[j] = (m >> j & 1) ? atomicAdd(&gp_base[gid[j] >> bw], 1u) : 0u;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (m >> j & 1)
                out_gid[pos[j]] = (uint32_t)gid[j];
        for (int s = 1; s < NS; s++) {
            long long va[4], vb[4] = {0, 0, 0, 0};
            load4_int(as.sa[s], as.sadt[s], ((uintptr_t)as.sa[s] % 16) == 0, r, c1, va);
            if (as.sop[s] == TDP_AGG_SUM_MUL_KMINUS)
                load4_int(as.sb[s], as.sbdt[s], ((uintptr_t)as.sb[s] % 16) == 0, r, c1, vb);
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (m >> j & 1)
                    out_val[(s - 1) * val_stride + pos[j]] =
                        as.sop[s] == TDP_AGG_SUM_MUL_KMINUS ? va[j] * (as.sk[s] - vb[j]) : va[j];
        }
    }
}

// One block per bucket b: dense table of the bucket's B gids in shared
// memory, then its non-empty gids in ascending order at the offset found by
// look-back over buckets 0..b-1.  Slot l of the table belongs to thread
// l % 256 in round l / 256 (conflict-free reads); ranks come from one ballot
// per round and a scan over the (round, warp) counts; the slot of every rank
// is kept in shared memory so that the groups are written with coalesced
// stores.
__global__ void __launch_bounds__(GP_THREADS) part_reduce_kernel(KeySet ks, AggSet as, DenseOut out, int bw,
                                                                 long long D, const unsigned *start,
                                                                 const uint32_t *gid, const long long *val,
                                                                 long long val_stride, long long cap,
                                                                 long long *d_ngroups,
                                                                 unsigned long long *tile_status,
                                                                 int32_t *d_status, uint32_t limit, int nb)
{
    constexpr int NW = GP_THREADS / 32;
    constexpr int MAX_ROUNDS = 4096 / GP_THREADS;
    extern __shared__ long long gp_acc[];
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    __shared__ unsigned s_cnt[MAX_ROUNDS * NW];
    __shared__ unsigned s_btot;
    __shared__ unsigned long long s_excl;
    const int NS = as.nslots;
    const int B = 1 << bw;
    uint16_t *s_idx = (uint16_t *)(gp_acc + (size_t)B * NS); // rank -> slot
    const int b = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid <= TDP_MAX_AGGS) {
        s_ops[tid] = slot_op(as, tid);
        s_init[tid] = slot_init(as, tid);
    }
    __syncthreads();
    for (int e = tid; e < B * NS; e += GP_THREADS)
        gp_acc[e] = s_init[e % NS];
    __syncthreads();

    // accumulate the bucket's segment, four elements a thread in flight (a gid
    // outside the bucket cannot come from the scatter; it is skipped, not used
    // as an index, and reported)
    bool bad = false;
    const unsigned lo = start[b], hi = start[b + 1];
    const unsigned gbase = (unsigned)b << bw;
    if (NS == 2) {
        const int op1 = s_ops[1];
        for (unsigned i0 = lo + tid; i0 < hi; i0 += 4 * GP_THREADS) {
            uint32_t g[4];
            long long v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned i = i0 + k * GP_THREADS;
                g[k] = i < hi ? gid[i] : 0xffffffffu;
                v[k] = i < hi ? val[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (g[k] != 0xffffffffu) {
                    if (g[k] - gbase >= (unsigned)B) { // not this bucket's: skipped and flagged
                        bad = true;
                        continue;
                    }
                    long long *a = gp_acc + (size_t)(g[k] - gbase) * 2;
                    atomicAdd((unsigned long long *)&a[0], 1ull);
                    acc_update(&a[1], op1, v[k]);
                }
        }
    } else {
        for (unsigned i0 = lo + tid; i0 < hi; i0 += 4 * GP_THREADS) {
            uint32_t g[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned i = i0 + k * GP_THREADS;
                g[k] = i < hi ? gid[i] : 0xffffffffu;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (g[k] == 0xffffffffu)
                    continue;
                if (g[k] - gbase >= (unsigned)B) {
                    bad = true;
                    continue;
                }
                const unsigned i = i0 + k * GP_THREADS;
                long long *a = gp_acc + (size_t)(g[k] - gbase) * NS;
                atomicAdd((unsigned long long *)&a[0], 1ull);
                for (int sl = 1; sl < NS; sl++)
                    acc_update(&a[sl], s_ops[sl], val[(sl - 1) * val_stride + i]);
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    __syncthreads();

    // ranks of the non-empty slots
    const int R = (B + GP_THREADS - 1) / GP_THREADS;
    const unsigned lt = lanemask_lt();
    for (int r = 0; r < R; r++) {
        const int l = r * GP_THREADS + tid;
        const unsigned bal = __ballot_sync(0xffffffffu, l < B && gp_acc[(size_t)l * NS] > 0);
        if (lane == 0)
            s_cnt[r * NW + warp] = __popc(bal);
    }
    __syncthreads();
    if (warp == 0) { // exclusive scan of the R x NW counts (at most 128)
        unsigned v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int e = lane * 4 + q;
            v[q] = e < R * NW ? s_cnt[e] : 0u;
            sum += v[q];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += u;
        }
        unsigned run = incl - sum;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int e = lane * 4 + q;
            if (e < R * NW)
                s_cnt[e] = run;
            run += v[q];
        }
        const unsigned btot = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned long long e = lookback_exclusive(tile_status, b, btot, limit, d_status);
        if (lane == 0) {
            s_btot = btot;
            s_excl = e;
            if (b == nb - 1) {
                const long long total = (long long)(e + btot);
                *d_ngroups = total;
                if (total > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    for (int r = 0; r < R; r++) {
        const int l = r * GP_THREADS + tid;
        const bool ne = l < B && gp_acc[(size_t)l * NS] > 0;
        const unsigned bal = __ballot_sync(0xffffffffu, ne);
        if (ne)
            s_idx[s_cnt[r * NW + warp] + __popc(bal & lt)] = (uint16_t)l;
    }
    __syncthreads();

    // coalesced output of the bucket's groups
    const long long excl = (long long)s_excl;
    const unsigned lim = (unsigned)max(0ll, min((long long)s_btot, cap - excl));
    for (unsigned i = tid; i < lim; i += GP_THREADS) {
        const int l = s_idx[i];
        const long long g = (long long)gbase + l;
        const long long pos = excl + i;
#pragma unroll
        for (int k = 0; k < TDP_MAX_KEYS; k++) { // static indices: the descriptors stay in parameter space
            if (k >= ks.n)
                break;
            const long long key = ks.n == 1 ? ks.lo[0] + g : ks.lo[k] + (g / ks.stride[k]) % ks.size[k];
            switch (out.key_dt[k]) {
            case TDP_I8: ((int8_t *)out.key_out[k])[pos] = (int8_t)key; break;
            case TDP_U8: ((uint8_t *)out.key_out[k])[pos] = (uint8_t)key; break;
            case TDP_I32: ((int32_t *)out.key_out[k])[pos] = (int32_t)key; break;
            default: ((long long *)out.key_out[k])[pos] = key; break;
            }
        }
#pragma unroll
        for (int a = 0; a < TDP_MAX_AGGS; a++)
            if (a < as.n)
                out.agg_out[a][pos] = agg_final(as, a, gp_acc + (size_t)l * NS);
    }
    (void)D;
}

// ------------------------------------------------------------------ host

// Count and scatter run on this grid (the chunks of rows must match).
static int part_grid() { return num_sms() * 2; }

size_t part_ws(long long n, long long D, int nslots)
{
    PartPlan pp;
    if (!part_plan(D, nslots, &pp))
        return 0;
    size_t b = 2 * align_up((size_t)(pp.nb + 1) * 4, 256);               // hist, start
    b += align_up((size_t)part_grid() * pp.nb * 4, 256);                 // block offsets within buckets
    b += align_up(16 + (size_t)pp.nb * 8, 256);                          // look-back words
    b += align_up((size_t)std::max(1ll, n) * 4, 256);                    // gids
    b += (size_t)(nslots - 1) * align_up((size_t)std::max(1ll, n) * 8, 256); // slot values
    return b;
}

tdp_status part_run(const PredSet &ps, const KeySet &ks, const AggSet &as, long long D, long long n,
                    const int32_t *sel, const int64_t *d_nsel, const DenseOut &out, long long capacity,
                    int64_t *d_ngroups, void *ws, int32_t *d_status, cudaStream_t s)
{
    PartPlan pp;
    if (!part_plan(D, as.nslots, &pp))
        return TDP_ERR_INVALID_ARG;
    const int nb = (int)pp.nb;
    const int G = part_grid();
    char *p = (char *)ws;
    unsigned *hist = (unsigned *)p;
    p += align_up((size_t)(nb + 1) * 4, 256);
    unsigned *start = (unsigned *)p;
    p += align_up((size_t)(nb + 1) * 4, 256);
    unsigned *boff = (unsigned *)p;
    p += align_up((size_t)G * nb * 4, 256);
    unsigned long long *lb = (unsigned long long *)(p + 16);
    cudaMemsetAsync(p, 0, 16 + (size_t)nb * 8, s);
    p += align_up(16 + (size_t)nb * 8, 256);
    uint32_t *gid = (uint32_t *)p;
    p += align_up((size_t)std::max(1ll, n) * 4, 256);
    long long *val = (long long *)p;
    const long long val_stride = (long long)(align_up((size_t)std::max(1ll, n) * 8, 256) / 8);
    cudaMemsetAsync(hist, 0, (size_t)nb * 4, s);

    // (the opt-in is set whatever the size: static shared memory adds to it)
    const size_t hsm = (size_t)nb * 4;
    const long long *dn = (const long long *)d_nsel;
    auto cnt = sel ? part_count_kernel<true> : part_count_kernel<false>;
    auto sct = sel ? part_scatter_kernel<true> : part_scatter_kernel<false>;
    if (cudaFuncSetAttribute(cnt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm) != cudaSuccess ||
        cudaFuncSetAttribute(sct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm) != cudaSuccess)
        return TDP_ERR_CUDA;
    if (n > 0)
        cnt<<<G, GS_THREADS, hsm, s>>>(ps, ks, n, sel, dn, pp.bw, nb, hist, boff, d_status);
    part_scan_kernel<<<1, 1024, 0, s>>>(hist, nb, start);
    if (n > 0)
        sct<<<G, GS_THREADS, hsm, s>>>(ps, ks, as, n, sel, dn, pp.bw, nb, start, boff, gid, val, val_stride);
    const size_t tsm = ((size_t)1 << pp.bw) * (as.nslots * 8 + 2); // table + rank -> slot index
    if (cudaFuncSetAttribute(part_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) !=
        cudaSuccess)
        return TDP_ERR_CUDA;
    part_reduce_kernel<<<nb, GP_THREADS, tsm, s>>>(ks, as, out, pp.bw, D, start, gid, val, val_stride, capacity,
                                                  (long long *)d_ngroups, lb, d_status, spin_limit(), nb);
    return launch_status();
}

} // namespace tdp
