// K7: group-join where the group key is the join key, over a rank code of
// the build keys.
//
// SELECT k, aggs(probe columns) FROM build JOIN probe ON build.key = probe.key
// WHERE build preds AND probe preds GROUP BY k ORDER BY k [, top-k by one
// aggregate], for unique build keys bounded by [lo, hi] (the column metadata
// of Sec. 2 that selects an operator strategy).  Sec. 2 (Data Encoding) keeps
// an order-preserving dictionary code per column; here the build side's key
// set is turned into exactly such a code on the device, and the code is the
// accumulator index:
//
//   1. build: every qualifying build row sets bit (key - lo) of a bitmap of
//      D = hi - lo + 1 bits, stored as words of 32 keys with a rank field
//      beside each word ({bits, rank}: 8 bytes per 32 keys, 3.75 MB for
//      D = 15M), by atomic ORs; the inserted rows are counted, and fewer set
//      bits than inserted rows means a duplicate build key.
//   2. rank (cooperative, one bounded grid barrier): an exclusive scan of
//      the words' popcounts writes each word's rank; the code of key k is
//      then rank[w] + popc(bits[w] below k's bit), a dense number in 0..B-1
//      in ascending key order (B build keys).  The same pass sets the B
//      accumulator rows to their initial values.
//   3. probe: every warp works alone on chunks of probe rows that lane 0
//      bulk-copies into the warp's two shared-memory buffers (completion on
//      the warp's own mbarrier), so the next chunk's columns are in flight
//      while the warp works on this one.  Phase A: predicates, then the
//      bitmap word of every qualifying key (one 8-byte load, L2-resident; all
//      of a lane's lookups in flight together); a hit sets the key's bit in a
//      second bitmap of the matched keys and is queued in the warp's own
//      shared-memory slots.  Phase B: the lanes take the queue, gather the
//      hits' aggregate inputs and add them into accumulator row `code` with
//      64-bit atomics (L2-resident: B x slots x 8 bytes).  No block barrier.
//   4. finalize: a cooperative hit-rank scan over the matched-key bitmap
//      gives every word its first output position; an output pass walks the
//      bits in order, which walks the keys in order, so the groups come out
//      sorted with no sort (key = lo + 32 w + bit, aggregates from row
//      rank + popc).  With a top-k request, blocks rank their shares of the
//      groups exactly behind a shared lower bound and one block merges their
//      candidates.
//
// The integer accumulation is exact and order-independent, so the result is
// bit-identical to join, then group-by, then top-k.
// Nothing is written per match and no partition or sort of the matches is
// needed; the per-row traffic is the probe-side columns.
#include <algorithm>
#include <cstring>

#include "filter_api.cuh"
#include "groupby.cuh"
#include "coop.cuh"
#include "topk.cuh"

namespace tdp {

constexpr int GJR_THREADS = 256;
constexpr int GJR_STEPS = 2;               // probe rows per thread per tile: 4 x GJR_STEPS

struct __align__(8) RankWord {
    uint32_t bits;
    uint32_t rank;
};

// Accumulator rows: `stride` int64 per code.  Slot 0 (COUNT) is stored only
// when an aggregate needs it (COUNT or AVG); otherwise slot s is stored at
// s - 1 and the matched-key bitmap alone says which groups exist.
struct AccLayout {
    int cs;     // first stored slot (0 or 1)
    int stride; // as.nslots - cs
};

__device__ __forceinline__ long long gj_final(const AggSet &as, int a, const long long *row, int cs)
{
    const int op = as.op[a];
    if (op == TDP_AGG_COUNT)
        return row[0];
    const long long s = row[as.slot[a] - cs];
    if (op == TDP_AGG_AVG) {
        const long long c = row[0];
        const long long sg = s > 0 ? 1 : (s < 0 ? -1 : 0);
        return (2 * s + sg * c) / (2 * c);
    }
    return s;
}

// ---------------------------------------------------------------- 1. build

// Mask (bit e = row r0 + e) of the rows r0 .. r0+15 (r0 % 16 == 0, rows < n)
// that satisfy predicate p.  A full group of an aligned column is read with
// 16-byte loads (one load holds 16 int8, 4 int32 or 2 int64 rows) and
// tested in the column's own width.
__device__ __forceinline__ unsigned pred_mask16(const PredSet &ps, int p, long long r0, long long n)
{
    const int dt = ps.dt[p];
    const unsigned neg = (unsigned)ps.neg[p];
    const bool full = r0 + 15 < n && ps.vec_ok[p];
    unsigned m = 0;
    if (dt == TDP_I64) {
        const long long lo = ps.lo[p];
        const unsigned long long span = (unsigned long long)(ps.hi[p] - lo);
        const long long *c = (const long long *)ps.col[p] + r0;
#pragma unroll
        for (int h = 0; h < 8; h++) {
            long long a, b;
            if (full) {
                const longlong2 v = __ldg((const longlong2 *)c + h);
                a = v.x, b = v.y;
            } else {
                a = r0 + 2 * h < n ? c[2 * h] : 0;
                b = r0 + 2 * h + 1 < n ? c[2 * h + 1] : 0;
            }
            m |= (range_holds64(a, lo, span, neg) | range_holds64(b, lo, span, neg) << 1) << (2 * h);
        }
        return m;
    }
    const int lo = (int)ps.lo[p];
    const unsigned span = (unsigned)((int)ps.hi[p] - lo);
    if (dt == TDP_I32) {
        const int32_t *c = (const int32_t *)ps.col[p] + r0;
#pragma unroll
        for (int h = 0; h < 4; h++) {
            int4 v;
            if (full) {
                v = __ldg((const int4 *)c + h);
            } else {
                v.x = r0 + 4 * h < n ? c[4 * h] : 0;
                v.y = r0 + 4 * h + 1 < n ? c[4 * h + 1] : 0;
                v.z = r0 + 4 * h + 2 < n ? c[4 * h + 2] : 0;
                v.w = r0 + 4 * h + 3 < n ? c[4 * h + 3] : 0;
            }
            m |= (range_holds32(v.x, lo, span, neg) | range_holds32(v.y, lo, span, neg) << 1 |
                  range_holds32(v.z, lo, span, neg) << 2 | range_holds32(v.w, lo, span, neg) << 3)
                 << (4 * h);
        }
        return m;
    }
    // int8 / uint8: four rows per 32-bit word with byte-wise SIMD.  For bytes,
    // (v - lo) mod 256 <= hi - lo (unsigned) holds exactly when lo <= v <= hi,
    // in the column's own signedness, because the span is below 256.
    const uint8_t *c = (const uint8_t *)ps.col[p] + r0;
    uint4 v;
    if (full) {
        v = __ldg((const uint4 *)c);
    } else {
        uint32_t w[4] = {0, 0, 0, 0};
        for (int e = 0; e < 16 && r0 + e < n; e++)
            w[e / 4] |= (uint32_t)c[e] << (8 * (e & 3));
        v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
    const uint32_t lo4 = ((uint32_t)lo & 0xffu) * 0x01010101u;
    const uint32_t sp4 = (span & 0xffu) * 0x01010101u;
#pragma unroll
    for (int h = 0; h < 4; h++) {
        const uint32_t x = __vcmpleu4(__vsub4(ww[h], lo4), sp4) & 0x01010101u;
        const uint32_t bits = ((x * 0x01020408u) >> 24) & 0xfu; // byte e -> bit e
        m |= (neg ? bits ^ 0xfu : bits) << (4 * h);
    }
    return m;
}

// 16 rows per thread: the predicate columns and the keys of all 16 rows are
// loaded before the first insert (one round trip instead of a chain).  The
// inserts are atomic ORs without a return value; the number of inserted rows
// goes to *d_rows, and the rank pass compares it with the number of set bits:
// fewer bits than rows means a key was inserted twice (a duplicate build key).
// Keys and [lo, hi] are int32 and D <= 2^31, so (unsigned)(key - lo) < D in
// 32-bit arithmetic is the bounds test.
constexpr int GJB_ROWS = 16;

__global__ void __launch_bounds__(256) gjr_build_kernel(PredSet ps, const int32_t *__restrict__ key, long long n,
                                                        const long long *d_n, int lo32, unsigned D32, RankWord *bm,
                                                        unsigned long long *d_rows, int32_t *d_status)
{
    if (d_n)
        n = min(*d_n, n);
    const bool kvec = ((uintptr_t)key % 16) == 0;
    const long long groups = (n + GJB_ROWS - 1) / GJB_ROWS;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned rows = 0;
    bool out_of_bounds = false;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < groups; gi += stride) {
        const long long r0 = gi * GJB_ROWS;
        const bool full = r0 + 15 < n;
        // the keys are loaded with the predicate columns (a full group almost
        // always holds a qualifying row), not after them
        int k[GJB_ROWS];
        if (full && kvec) {
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int4 kk = __ldg((const int4 *)(key + r0) + h);
                k[4 * h] = kk.x, k[4 * h + 1] = kk.y, k[4 * h + 2] = kk.z, k[4 * h + 3] = kk.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < GJB_ROWS; q++)
                k[q] = r0 + q < n ? key[r0 + q] : 0;
        }
        unsigned m = full ? 0xffffu : (1u << (unsigned)(n - r0)) - 1u;
        for (int p = 0; p < ps.n; p++)
            m &= pred_mask16(ps, p, r0, n);
#pragma unroll
        for (int q = 0; q < GJB_ROWS; q++) {
            if (!(m >> q & 1u))
                continue;
            const unsigned d = (unsigned)(k[q] - lo32);
            if (d >= D32) { // a build key outside its declared bounds
                out_of_bounds = true;
                continue;
            }
            atomicOr(&bm[d >> 5].bits, 1u << (d & 31u)); // result unused: a reduction
            rows++;
        }
    }
    if (out_of_bounds)
        set_status(d_status, TDP_ERR_OVERFLOW);
    // inserted rows: one atomic per warp (every thread of the grid gets here)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        rows += __shfl_xor_sync(0xffffffffu, rows, o);
    if ((threadIdx.x & 31) == 0 && rows)
        atomicAdd(d_rows, (unsigned long long)rows);
}

// ----------------------------------------------------------------- 2. rank

// Cooperative passes over the bitmap words (the rank pass and the finalize):
// thread t of block b owns the WPT consecutive words starting at
// (b * 256 + t) * WPT, so one block scan of the threads' counts orders all of
// the block's words.  Every block publishes its total, waits once on a
// bounded grid-wide barrier for all blocks to have counted, and starts from
// the sum of the totals of the blocks before it: no chain of tiles.

// Rank pass: bm[w].rank = set bits before word w; accumulator rows of the
// build keys set to their initial values; B (all set bits) to *d_nkeys.
// d_rows: the inserted build rows (more rows than bits: a duplicate build
// key).  A block owns `rounds`
// consecutive spans of 256 x WPT words (more than one only when the domain
// has more words than the resident blocks cover).
template <int WPT>
__global__ void __launch_bounds__(GJR_THREADS) gjr_rank_kernel(RankWord *bm, long long W, int rounds, AggSet as,
                                                               AccLayout al, long long *acc,
                                                               unsigned long long *d_nkeys,
                                                               const unsigned long long *d_rows,
                                                               unsigned long long *totals, unsigned *barrier,
                                                               int32_t *d_status, uint32_t limit)
{
    __shared__ unsigned long long s_red[GJR_THREADS / 32];
    __shared__ unsigned s_warp[GJR_THREADS / 32];
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    if (threadIdx.x <= TDP_MAX_AGGS)
        s_init[threadIdx.x] = slot_init(as, threadIdx.x);
    const long long span = (long long)GJR_THREADS * WPT;
    const long long b0 = (long long)blockIdx.x * rounds * span;
    uint32_t b[WPT];
    unsigned long long c = 0;
    for (int r = 0; r < rounds; r++) {
        const long long w0 = b0 + r * span + (long long)threadIdx.x * WPT;
#pragma unroll
        for (int i = 0; i < WPT; i++)
            b[i] = w0 + i < W ? bm[w0 + i].bits : 0u;
#pragma unroll
        for (int i = 0; i < WPT; i++)
            c += __popc(b[i]);
    }
    const unsigned long long total = block_sum(c, s_red);
    const unsigned long long prefix = coop_block_prefix(total, s_red, totals, barrier, limit, d_status);
    unsigned long long run = prefix;
    for (int r = 0; r < rounds; r++) {
        const long long w0 = b0 + r * span + (long long)threadIdx.x * WPT;
        unsigned cr = 0;
#pragma unroll
        for (int i = 0; i < WPT; i++) {
            b[i] = w0 + i < W ? bm[w0 + i].bits : 0u;
            cr += __popc(b[i]);
        }
        unsigned tot;
        unsigned rk = (unsigned)(run + block_excl_scan(cr, s_warp, &tot));
#pragma unroll
        for (int i = 0; i < WPT; i++)
            if (w0 + i < W) {
                bm[w0 + i].rank = rk;
                rk += __popc(b[i]);
            }
        run += tot;
        __syncthreads(); // s_warp reused by the next round's scan
    }
    // initial values of the block's accumulator rows (contiguous codes)
    const int S = al.stride;
    long long *a0 = acc + (long long)prefix * S;
    for (long long j = threadIdx.x; j < (long long)total * S; j += GJR_THREADS)
        a0[j] = s_init[al.cs + (int)(j % S)];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *d_nkeys = prefix + total;
        if (*d_rows != prefix + total)
            set_status(d_status, TDP_ERR_DUP_BUILD_KEY);
    }
}

// ---------------------------------------------------------------- 3. probe

// Aggregate input of a probe row read from global memory (read once:
// evict-first in L2).
__device__ __forceinline__ long long gather_int(const void *p, int dt, long long row, uint64_t pol)
{
    switch (dt) {
    case TDP_I8: return ((const int8_t *)p)[row];
    case TDP_U8: return ((const uint8_t *)p)[row];
    case TDP_I32: return ldg_hint((const int32_t *)p + row, pol);
    default: return ldg_hint((const long long *)p + row, pol);
    }
}

// Every warp works on its own: chunks of GJR_CHUNK rows in grid-stride order,
// lane rows c*GJR_CHUNK + j*128 + 4*lane + 0..3 (j < GJR_STEPS), read with
// 16-byte (4-row) vector loads.  Phase A: predicates, then the bitmap word of
// every qualifying key (all of the lane's lookups in flight together); a hit
// sets the key's bit in the matched-key bitmap and is queued in the warp's
// own shared-memory slots (ballot ranks).  Phase B: the warp's lanes take the
// queue, gather the aggregate inputs and add them into accumulator row
// `code`.  No block-wide barrier.  NSMAX: accumulator slots the kernel is
// compiled for (COUNT + sums).
constexpr int GJR_CHUNK = 128 * GJR_STEPS;
constexpr int GJR_PROBE_THREADS = 256;

template <int NSMAX>
__global__ void __launch_bounds__(GJR_PROBE_THREADS, 4)
    gjr_probe_direct_kernel(PredSet ps, const int32_t *__restrict__ key, int key_vec, long long n_host,
                     const long long *d_n, int lo32, unsigned D32, const RankWord *bm, uint32_t *hitw, AggSet as,
                     AccLayout al, long long *acc, unsigned long long *d_nmatch)
{
    constexpr int NB = 2;                      // queue entries per lane in flight in phase B
    constexpr int VS = NSMAX <= 4 ? NSMAX : 1; // slots gathered ahead of the atomics
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    // per-warp hit queues: row within the chunk, and code
    __shared__ uint16_t s_q[GJR_PROBE_THREADS / 32][GJR_CHUNK];
    __shared__ uint32_t s_c[GJR_PROBE_THREADS / 32][GJR_CHUNK];
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x <= TDP_MAX_AGGS)
        s_ops[threadIdx.x] = slot_op(as, threadIdx.x);
    __syncthreads();
    const int NS = as.nslots;
    const bool count = al.cs == 0;
    const uint64_t stream_pol = l2_evict_first(), table_pol = l2_evict_last();
    const unsigned lt = lanemask_lt();
    const long long nchunks = (n + GJR_CHUNK - 1) / GJR_CHUNK;
    const long long wstride = (long long)gridDim.x * (GJR_PROBE_THREADS / 32);
    unsigned long long matches = 0;
    for (long long c = (long long)blockIdx.x * (GJR_PROBE_THREADS / 32) + warp; c < nchunks; c += wstride) {
        const long long base = c * GJR_CHUNK;
        // ---- phase A
        unsigned msk[GJR_STEPS];
#pragma unroll
        for (int j = 0; j < GJR_STEPS; j++) {
            const long long r = base + j * 128 + 4 * lane;
            msk[j] = r + 3 < n ? 0xfu : (r + 2 < n ? 0x7u : (r + 1 < n ? 0x3u : (r < n ? 0x1u : 0u)));
        }
        int k[GJR_STEPS * 4];
#pragma unroll
        for (int j = 0; j < GJR_STEPS; j++) {
            const long long r = base + j * 128 + 4 * lane;
            if (key_vec && r + 3 < n) {
                const uint4 kk = ldg16_hint((const uint32_t *)(key + r), stream_pol);
                k[4 * j] = (int)kk.x, k[4 * j + 1] = (int)kk.y, k[4 * j + 2] = (int)kk.z, k[4 * j + 3] = (int)kk.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    k[4 * j + e] = r + e < n ? key[r + e] : 0;
            }
        }
        for (int p = 0; p < ps.n; p++) {
            long long v[GJR_STEPS][4];
#pragma unroll
            for (int j = 0; j < GJR_STEPS; j++)
                load4_int(ps.col[p], ps.dt[p], ps.vec_ok[p], base + j * 128 + 4 * lane, n, v[j]);
            const unsigned long long span = (unsigned long long)(ps.hi[p] - ps.lo[p]);
#pragma unroll
            for (int j = 0; j < GJR_STEPS; j++)
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (!range_holds64(v[j][e], ps.lo[p], span, (unsigned)ps.neg[p]))
                        msk[j] &= ~(1u << e);
        }
        unsigned long long wv[GJR_STEPS * 4];
        unsigned dd[GJR_STEPS * 4];
        unsigned look = 0;
#pragma unroll
        for (int q = 0; q < GJR_STEPS * 4; q++) {
            dd[q] = (unsigned)(k[q] - lo32);
            if ((msk[q / 4] >> (q & 3) & 1u) && dd[q] < D32) {
                look |= 1u << q;
                wv[q] = ldg_hint((const unsigned long long *)(bm + (dd[q] >> 5)), table_pol);
            }
        }
        unsigned qbase = 0;
#pragma unroll
        for (int q = 0; q < GJR_STEPS * 4; q++) {
            bool hit = false;
            uint32_t code = 0;
            if (look >> q & 1u) {
                const uint32_t bits = (uint32_t)wv[q];
                const unsigned bp = dd[q] & 31u;
                if ((bits >> bp) & 1u) {
                    hit = true;
                    code = (uint32_t)(wv[q] >> 32) + __popc(bits & ((1u << bp) - 1u));
                    atomicOr(&hitw[dd[q] >> 5], 1u << bp);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const unsigned pos = qbase + __popc(bal & lt);
                s_q[warp][pos] = (uint32_t)((q / 4) * 128 + 4 * lane + (q & 3));
                s_c[warp][pos] = code;
            }
            qbase += __popc(bal);
        }
        __syncwarp();
        // ---- phase B
        matches += qbase; // lane 0's count is the warp's
        for (unsigned i0 = 0; i0 < qbase; i0 += 32 * NB) {
            long long row[NB];
            uint32_t cd[NB];
            long long va[NB][VS], vb[NB][VS];
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const unsigned i = i0 + lane + 32 * u;
                row[u] = i < qbase ? base + s_q[warp][i] : -1;
                cd[u] = i < qbase ? s_c[warp][i] : 0u;
                if constexpr (NSMAX <= 4) {
                    if (row[u] >= 0) {
#pragma unroll
                        for (int sl = 1; sl < VS; sl++) {
                            if (sl >= NS)
                                break;
                            va[u][sl] = gather_int(as.sa[sl], as.sadt[sl], row[u], stream_pol);
                            vb[u][sl] = as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS
                                            ? gather_int(as.sb[sl], as.sbdt[sl], row[u], stream_pol)
                                            : 0;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < NB; u++) {
                if (row[u] < 0)
                    continue;
                long long *arow = acc + (long long)cd[u] * al.stride; // slot s at arow[s - cs]
                if (count)
                    atomicAdd((unsigned long long *)arow, 1ull);
                if constexpr (NSMAX <= 4) {
#pragma unroll
                    for (int sl = 1; sl < VS; sl++) {
                        if (sl >= NS)
                            break;
                        long long v = va[u][sl];
                        if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                            v *= as.sk[sl] - vb[u][sl];
                        acc_update(arow + (sl - al.cs), s_ops[sl], v);
                    }
                } else {
                    for (int sl = 1; sl < NS; sl++) {
                        long long v = gather_int(as.sa[sl], as.sadt[sl], row[u], stream_pol);
                        if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                            v *= as.sk[sl] - gather_int(as.sb[sl], as.sbdt[sl], row[u], stream_pol);
                        acc_update(arow + (sl - al.cs), s_ops[sl], v);
                    }
                }
            }
        }
        __syncwarp(); // the warp's queue is free for the next chunk
    }
    if (lane == 0 && matches && d_nmatch)
        atomicAdd(d_nmatch, matches);
}

// The same probe with each warp's chunks staged in shared memory: lane 0
// bulk-copies the key and predicate columns of the warp's next chunk into
// the other of the warp's two buffers (completion on the warp's own
// mbarrier) before the warp works on the current one, so the column stream
// stays in flight while the warp waits on its lookups and gathers.  Chunks
// that are ragged or whose columns are not 16-byte aligned are loaded by the
// lanes instead.  Still no block-wide barrier after the set-up.
constexpr int GJR_MAX_STAGE = 1 + TDP_MAX_PREDS;
constexpr int GJR_STAGE_MAX_ROW = 24; // bytes of staged columns per row (two buffers per warp)

struct GJRStage {
    const void *col[GJR_MAX_STAGE]; // [0] the probe key, then each distinct predicate column
    int32_t size[GJR_MAX_STAGE];
    int32_t n;
    int32_t aligned;             // every staged column 16-byte aligned
    int32_t pred[TDP_MAX_PREDS]; // stage index of predicate p's column
};

// (Measured: pipelining the warp's chunks -- chunk i's lookups in flight
// while chunk i-1's hits are gathered, with two hit queues per warp -- cost
// one resident block per SM for the second queue and ran slower, 314 vs
// 289 us on the 60M-row probe.)
template <int NSMAX>
__global__ void __launch_bounds__(GJR_PROBE_THREADS, 4)
    gjr_probe_kernel(PredSet ps, GJRStage sg, long long n_host, const long long *d_n, int lo32, unsigned D32,
                     const RankWord *bm, uint32_t *hitw, AggSet as, AccLayout al, long long *acc,
                     unsigned long long *d_nmatch, int32_t *d_status, uint32_t limit)
{
    constexpr int NB = 2;                      // queue entries per lane in flight in phase B
    constexpr int VS = NSMAX <= 4 ? NSMAX : 1; // slots gathered ahead of the atomics
    constexpr int WARPS = GJR_PROBE_THREADS / 32;
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    extern __shared__ __align__(128) unsigned char gjr_smem[]; // [warp][2][GJR_CHUNK x row bytes]
    __shared__ __align__(8) uint64_t s_bar[WARPS][2];
    __shared__ uint16_t s_q[WARPS][1][GJR_CHUNK];
    __shared__ uint32_t s_c[WARPS][1][GJR_CHUNK];
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    __shared__ uint32_t s_off[GJR_MAX_STAGE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t row_bytes = 0;
    for (int c = 0; c < sg.n; c++)
        row_bytes += sg.size[c];
    if (threadIdx.x <= TDP_MAX_AGGS)
        s_ops[threadIdx.x] = slot_op(as, threadIdx.x);
    if (threadIdx.x == 0) {
        uint32_t off = 0;
        for (int c = 0; c < sg.n; c++) {
            s_off[c] = off;
            off += GJR_CHUNK * sg.size[c];
        }
    }
    if (lane == 0) {
        mbar_init(&s_bar[warp][0], 1);
        mbar_init(&s_bar[warp][1], 1);
    }
    __syncthreads();
    const int NS = as.nslots;
    const bool count = al.cs == 0;
    const uint64_t stream_pol = l2_evict_first(), table_pol = l2_evict_last();
    const unsigned lt = lanemask_lt();
    const long long nchunks = (n + GJR_CHUNK - 1) / GJR_CHUNK;
    const long long wstride = (long long)gridDim.x * WARPS;
    unsigned char *wbuf = gjr_smem + (size_t)warp * 2 * GJR_CHUNK * row_bytes;
    auto bulk_ok = [&](long long c) { return sg.aligned && (c + 1) * GJR_CHUNK <= n; };
    auto issue = [&](long long c, int b) { // lane 0 only
        unsigned char *buf = wbuf + (size_t)b * GJR_CHUNK * row_bytes;
        fence_proxy_async_smem(); // the lanes' earlier reads of this buffer come first
        mbar_arrive_expect_tx(&s_bar[warp][b], GJR_CHUNK * row_bytes);
        for (int k = 0; k < sg.n; k++)
            bulk_load_hint(buf + s_off[k], (const char *)sg.col[k] + (size_t)c * GJR_CHUNK * sg.size[k],
                           GJR_CHUNK * sg.size[k], &s_bar[warp][b], stream_pol);
    };
    // gathers and atomics of one queued chunk (rows base + s_q)
    auto drain = [&](int qb, unsigned qn, long long base) {
        for (unsigned i0 = 0; i0 < qn; i0 += 32 * NB) {
            long long row[NB];
            uint32_t cd[NB];
            long long va[NB][VS], vb[NB][VS];
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const unsigned i = i0 + lane + 32 * u;
                row[u] = i < qn ? base + s_q[warp][qb][i] : -1;
                cd[u] = i < qn ? s_c[warp][qb][i] : 0u;
                if constexpr (NSMAX <= 4) {
                    if (row[u] >= 0) {
#pragma unroll
                        for (int sl = 1; sl < VS; sl++) {
                            if (sl >= NS)
                                break;
                            va[u][sl] = gather_int(as.sa[sl], as.sadt[sl], row[u], stream_pol);
                            vb[u][sl] = as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS
                                            ? gather_int(as.sb[sl], as.sbdt[sl], row[u], stream_pol)
                                            : 0;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < NB; u++) {
                if (row[u] < 0)
                    continue;
                long long *arow = acc + (long long)cd[u] * al.stride; // slot s at arow[s - cs]
                if (count)
                    atomicAdd((unsigned long long *)arow, 1ull);
                if constexpr (NSMAX <= 4) {
#pragma unroll
                    for (int sl = 1; sl < VS; sl++) {
                        if (sl >= NS)
                            break;
                        long long v = va[u][sl];
                        if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                            v *= as.sk[sl] - vb[u][sl];
                        acc_update(arow + (sl - al.cs), s_ops[sl], v);
                    }
                } else {
                    for (int sl = 1; sl < NS; sl++) {
                        long long v = gather_int(as.sa[sl], as.sadt[sl], row[u], stream_pol);
                        if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                            v *= as.sk[sl] - gather_int(as.sb[sl], as.sbdt[sl], row[u], stream_pol);
                        acc_update(arow + (sl - al.cs), s_ops[sl], v);
                    }
                }
            }
        }
    };
    const long long c0 = (long long)blockIdx.x * WARPS + warp;
    if (lane == 0 && c0 < nchunks && bulk_ok(c0))
        issue(c0, 0);
    bool late = false;
    unsigned long long matches = 0;
    uint32_t phase = 0;      // bit b: parity of buffer b's next phase
    int it = 0;
    for (long long c = c0; c < nchunks; c += wstride, it++) {
        const int b = it & 1;
        unsigned char *buf = wbuf + (size_t)b * GJR_CHUNK * row_bytes;
        const long long cn = c + wstride;
        if (lane == 0 && cn < nchunks && bulk_ok(cn))
            issue(cn, b ^ 1); // that buffer was consumed in the previous iteration
        const long long base = c * GJR_CHUNK;
        if (bulk_ok(c)) {
            late |= !mbar_wait(&s_bar[warp][b], (phase >> b) & 1u, limit);
            phase ^= 1u << b;
        } else {
            for (int k = 0; k < sg.n; k++) {
                unsigned char *d = buf + s_off[k];
                for (int i = lane; i < GJR_CHUNK; i += 32) {
                    if (base + i >= n)
                        break;
                    switch (sg.size[k]) {
                    case 8: ((long long *)d)[i] = ((const long long *)sg.col[k])[base + i]; break;
                    case 4: ((int32_t *)d)[i] = ((const int32_t *)sg.col[k])[base + i]; break;
                    default: d[i] = ((const uint8_t *)sg.col[k])[base + i]; break;
                    }
                }
            }
            __syncwarp();
        }
        // ---- chunk c: predicates, then its lookups go out
        const long long left = n - base; // > 0
        unsigned msk[GJR_STEPS];
#pragma unroll
        for (int j = 0; j < GJR_STEPS; j++) {
            const long long r = j * 128 + 4 * lane;
            msk[j] = r + 3 < left ? 0xfu : (r + 2 < left ? 0x7u : (r + 1 < left ? 0x3u : (r < left ? 0x1u : 0u)));
        }
        for (int p = 0; p < ps.n; p++)
            pred_test_smem<GJR_STEPS>(ps, p, buf + s_off[sg.pred[p]], 4 * lane, msk);
        const int32_t *skey = (const int32_t *)buf; // stage 0 at offset 0
        unsigned long long wv[GJR_STEPS * 4];
        unsigned dd[GJR_STEPS * 4];
        unsigned look = 0;
#pragma unroll
        for (int j = 0; j < GJR_STEPS; j++) {
            const int4 k4 = *(const int4 *)(skey + j * 128 + 4 * lane);
            const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int q = j * 4 + e;
                dd[q] = (unsigned)(kk[e] - lo32);
                if ((msk[j] >> e & 1u) && dd[q] < D32) {
                    look |= 1u << q;
                    wv[q] = ldg_hint((const unsigned long long *)(bm + (dd[q] >> 5)), table_pol);
                }
            }
        }
        // ---- chunk c: hits to the queue (one warp scan of the lanes' counts)
        unsigned hm = 0;
#pragma unroll
        for (int q = 0; q < GJR_STEPS * 4; q++)
            if ((look >> q & 1u) && (((uint32_t)wv[q] >> (dd[q] & 31u)) & 1u))
                hm |= 1u << q;
        const unsigned nh = __popc(hm);
        unsigned incl = nh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += u;
        }
        const unsigned qbase = __shfl_sync(0xffffffffu, incl, 31);
        unsigned pos = incl - nh;
#pragma unroll
        for (int q = 0; q < GJR_STEPS * 4; q++)
            if (hm >> q & 1u) {
                const uint32_t bits = (uint32_t)wv[q];
                const unsigned bp = dd[q] & 31u;
                s_q[warp][0][pos] = (uint16_t)((q / 4) * 128 + 4 * lane + (q & 3));
                s_c[warp][0][pos] = (uint32_t)(wv[q] >> 32) + __popc(bits & ((1u << bp) - 1u));
                atomicOr(&hitw[dd[q] >> 5], 1u << bp);
                pos++;
            }
        matches += qbase; // lane 0's count is the warp's
        __syncwarp(); // chunk c's queue written
        // ---- chunk c: gathers and atomics of its hits
        drain(0, qbase, base);
        __syncwarp(); // the queue and the buffer are free for the next chunk
    }
    if (late)
        set_status(d_status, TDP_ERR_TIMEOUT);
    if (lane == 0 && matches && d_nmatch)
        atomicAdd(d_nmatch, matches);
}

// ------------------------------------------------------------- 4. finalize

// The exact top k (value desc, key asc, k <= 16) of `count` elements get(i)
// by one block, into s_best[0..k) (missing entries hold the worst value).
// Every thread keeps the largest of its elements; the k-th largest of those
// 256 maxima is reached by at least k elements, so only elements at or above
// it can be among the k best: those (a few more than k unless values tie)
// are ranked exactly by warp lists, or, past 256 of them, all elements are.
template <typename F>
__device__ __forceinline__ void block_topk(long long count, F get, int k, VK *s_best)
{
    __shared__ long long s_sort[GJR_THREADS];
    __shared__ VK s_cand[GJR_THREADS];
    __shared__ unsigned s_nc;
    constexpr int U = 8; // elements in flight per thread
    long long vmax = VK_WORST_V;
    bool has = false;
    for (long long i0 = threadIdx.x; i0 < count; i0 += (long long)GJR_THREADS * U) {
        long long v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = i0 + (long long)u * GJR_THREADS;
            v[u] = i < count ? get(i).v : VK_WORST_V;
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (i0 + (long long)u * GJR_THREADS < count) {
                vmax = has ? max(vmax, v[u]) : v[u];
                has = true;
            }
    }
    s_sort[threadIdx.x] = has ? vmax : VK_WORST_V;
    if (threadIdx.x == 0)
        s_nc = 0;
    __syncthreads();
    for (int k2 = 2; k2 <= GJR_THREADS; k2 <<= 1)
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            const int t = threadIdx.x, o = t ^ j;
            if (o > t) {
                const long long a0 = s_sort[t], a1 = s_sort[o];
                const bool desc = (t & k2) == 0;
                if (desc ? a0 < a1 : a0 > a1) {
                    s_sort[t] = a1;
                    s_sort[o] = a0;
                }
            }
            __syncthreads();
        }
    const long long T = s_sort[k - 1];
    for (long long i0 = threadIdx.x; i0 < count; i0 += (long long)GJR_THREADS * U) {
        VK c[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = i0 + (long long)u * GJR_THREADS;
            c[u] = i < count ? get(i) : VK{VK_WORST_V, VK_WORST_K};
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (i0 + (long long)u * GJR_THREADS < count && c[u].v >= T) {
                const unsigned j = atomicAdd(&s_nc, 1u);
                if (j < GJR_THREADS)
                    s_cand[j] = c[u];
            }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nc = s_nc;
    WarpList l;
    wl_init(l);
    if (nc <= GJR_THREADS) {
        for (unsigned b0 = warp * 32; b0 < nc; b0 += GJR_THREADS) {
            const unsigned i = b0 + lane;
            const VK c = i < nc ? s_cand[i] : VK{VK_WORST_V, VK_WORST_K};
            wl_offer(l, i < nc, c.v, c.k, k);
        }
    } else {
        for (long long b0 = warp * 32; b0 < count; b0 += GJR_THREADS) {
            const long long i = b0 + lane;
            const bool ok = i < count;
            const VK c = ok ? get(i) : VK{VK_WORST_V, VK_WORST_K};
            wl_offer(l, ok, c.v, c.k, k);
        }
    }
    block_merge(l, k, s_best);
    __syncthreads();
}

// Hit-rank pass (cooperative, like the rank pass) over the matched-key
// bitmap: hrank[w] = matched keys before word w; the group count to
// *d_ngroups (TDP_ERR_CAPACITY when it exceeds cap).
template <int WPT>
__global__ void __launch_bounds__(GJR_THREADS) gjr_hitrank_kernel(const uint32_t *hitw, long long W, int rounds,
                                                                  uint32_t *hrank, long long cap,
                                                                  long long *d_ngroups, unsigned long long *totals,
                                                                  unsigned *barrier, int32_t *d_status,
                                                                  uint32_t limit)
{
    __shared__ unsigned long long s_red[GJR_THREADS / 32];
    __shared__ unsigned s_warp[GJR_THREADS / 32];
    const long long span = (long long)GJR_THREADS * WPT;
    const long long b0 = (long long)blockIdx.x * rounds * span;
    uint32_t h[WPT];
    unsigned long long c = 0;
    for (int r = 0; r < rounds; r++) {
        const long long w0 = b0 + r * span + (long long)threadIdx.x * WPT;
#pragma unroll
        for (int i = 0; i < WPT; i++)
            h[i] = w0 + i < W ? hitw[w0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < WPT; i++)
            c += __popc(h[i]);
    }
    const unsigned long long total = block_sum(c, s_red);
    const unsigned long long prefix = coop_block_prefix(total, s_red, totals, barrier, limit, d_status);
    unsigned long long run = prefix;
    for (int r = 0; r < rounds; r++) {
        const long long w0 = b0 + r * span + (long long)threadIdx.x * WPT;
        unsigned cr = 0;
#pragma unroll
        for (int i = 0; i < WPT; i++) {
            h[i] = w0 + i < W ? hitw[w0 + i] : 0u;
            cr += __popc(h[i]);
        }
        unsigned tot;
        unsigned rk = (unsigned)(run + block_excl_scan(cr, s_warp, &tot));
#pragma unroll
        for (int i = 0; i < WPT; i++)
            if (w0 + i < W) {
                hrank[w0 + i] = rk;
                rk += __popc(h[i]);
            }
        run += tot;
        __syncthreads(); // s_warp reused by the next round's scan
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *d_ngroups = (long long)(prefix + total);
        if ((long long)(prefix + total) > cap)
            set_status(d_status, TDP_ERR_CAPACITY);
    }
}

// Output pass: each warp takes 32 consecutive words, lane i loading word i's
// bits, rank, matched bits and hit rank (coalesced).  Then, 8 words at a
// time, the words are broadcast and lane j takes the key of bit j in each:
// a matched key's group goes to position hrank + (matched keys below it in
// the word) from accumulator row rank + (build keys below it), so the lanes
// of a word read consecutive rows and write consecutive positions, with up
// to 8 rows in flight per lane.  NA: aggregates compiled for (>= as.n).
constexpr int GJR_OUT_GROUP = 8;

template <int NA>
__global__ void __launch_bounds__(GJR_THREADS) gjr_output_kernel(const RankWord *bm, const uint32_t *hitw,
                                                                 const uint32_t *hrank, long long W, long long lo,
                                                                 AggSet as, AccLayout al, const long long *acc,
                                                                 int32_t *out_keys, DenseOut out, long long cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const long long warps = (long long)gridDim.x * (GJR_THREADS / 32);
    const int na = as.n;
    for (long long w0 = ((long long)blockIdx.x * (GJR_THREADS / 32) + (threadIdx.x >> 5)) * 32; w0 < W;
         w0 += warps * 32) {
        const long long wl = w0 + lane;
        const bool in = wl < W;
        const RankWord e = in ? bm[wl] : RankWord{0u, 0u};
        const uint32_t hw = in ? hitw[wl] : 0u;
        const uint32_t hr = in ? hrank[wl] : 0u;
        unsigned busy = __ballot_sync(0xffffffffu, hw != 0u); // words with groups
        while (busy) {
            int q[GJR_OUT_GROUP];
#pragma unroll
            for (int g = 0; g < GJR_OUT_GROUP; g++) {
                q[g] = busy ? __ffs(busy) - 1 : -1;
                busy &= busy - 1;
            }
            long long v[GJR_OUT_GROUP][NA];
            long long pos[GJR_OUT_GROUP];
#pragma unroll
            for (int g = 0; g < GJR_OUT_GROUP; g++) {
                const int src = q[g] < 0 ? 0 : q[g];
                const uint32_t bits = __shfl_sync(0xffffffffu, e.bits, src);
                const uint32_t rank = __shfl_sync(0xffffffffu, e.rank, src);
                const uint32_t h = __shfl_sync(0xffffffffu, hw, src);
                const uint32_t r0 = __shfl_sync(0xffffffffu, hr, src);
                pos[g] = -1;
                if (q[g] >= 0 && ((h >> lane) & 1u)) {
                    pos[g] = (long long)r0 + __popc(h & lt);
                    const long long *row = acc + ((long long)rank + __popc(bits & lt)) * al.stride;
#pragma unroll
                    for (int a = 0; a < NA; a++)
                        if (a < na)
                            v[g][a] = gj_final(as, a, row, al.cs);
                }
            }
#pragma unroll
            for (int g = 0; g < GJR_OUT_GROUP; g++) {
                if (pos[g] < 0 || pos[g] >= cap)
                    continue;
                out_keys[pos[g]] = (int32_t)(lo + 32 * (w0 + q[g]) + lane);
#pragma unroll
                for (int a = 0; a < NA; a++)
                    if (a < na)
                        out.agg_out[a][pos[g]] = v[g][a];
            }
        }
    }
}

// Top-k pass over the written groups: block b ranks its contiguous share
// exactly (block_topk), writes its k best to cand[b * k] and raises the
// shared lower bound with its k-th best (at most the global k-th best).
__global__ void __launch_bounds__(GJR_THREADS) gjr_topk_blocks_kernel(const long long *vals, const int32_t *keys,
                                                                      const long long *d_ngroups, long long cap,
                                                                      int k, VK *cand, unsigned long long *bound)
{
    __shared__ VK s_best[TK_MAXK];
    const long long n = min(*d_ngroups, cap);
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long f = min(n, (long long)blockIdx.x * per);
    const long long cnt = min(n, f + per) - f;
    block_topk(cnt, [&](long long i) { return VK{vals[f + i], keys[f + i]}; }, k, s_best);
    if (threadIdx.x < k)
        cand[(size_t)blockIdx.x * k + threadIdx.x] = s_best[threadIdx.x];
    if (threadIdx.x == 0 && s_best[k - 1].k != VK_WORST_K)
        atomicMax(bound, enc_v(s_best[k - 1].v));
}

// The top k (value desc, key asc) of the per-block candidates: only those at
// or above the bound can be among them; min(k, groups) results.
__global__ void __launch_bounds__(GJR_THREADS) gjr_topk_final_kernel(const VK *cand, long long ncand, int k,
                                                                     const unsigned long long *bound,
                                                                     const long long *d_ngroups, long long cap,
                                                                     long long *out_vals, int32_t *out_keys,
                                                                     long long *d_k)
{
    __shared__ VK s_best[TK_MAXK];
    const long long gb = dec_v(*bound);
    block_topk(ncand, [&](long long i) {
        const VK c = cand[i];
        return (c.k != VK_WORST_K && c.v >= gb) ? c : VK{VK_WORST_V, VK_WORST_K};
    }, k, s_best);
    const long long m = min((long long)k, min(*d_ngroups, cap));
    if (threadIdx.x < m) {
        out_vals[threadIdx.x] = s_best[threadIdx.x].v;
        out_keys[threadIdx.x] = s_best[threadIdx.x].k;
    }
    if (threadIdx.x == 0 && d_k)
        *d_k = m;
}

// ----------------------------------------------------------------- host

struct GjrLayout {
    size_t counters, bitmap, hits, hrank, totals_rank, totals_hit, acc, cand, total;
    long long W, max_keys;
    int Gmax;    // most blocks a cooperative pass can have
    int topk_blocks; // blocks of the top-k pass
};

static GjrLayout gjr_layout(long long n_build, long long D, int naggs, int topk)
{
    GjrLayout L;
    L.W = (D + 31) / 32;
    // the cooperative passes have at most as many blocks as are resident at
    // once: 2048 threads per SM
    L.Gmax = (int)std::max(1ll, std::min<long long>((L.W + GJR_THREADS - 1) / GJR_THREADS, 8ll * num_sms()));
    L.topk_blocks = 4 * num_sms();
    L.max_keys = std::max(0ll, std::min(n_build, D));
    const size_t kk = (size_t)std::max(0, topk);
    size_t off = 0;
    // [0] build keys, [1] rank barrier, [2] hit-rank barrier, [3] top-k bound
    // (0: none), [4] inserted build rows, [5] joined rows
    L.counters = off;
    off += 256;
    L.bitmap = off;
    off = align_up(off + (size_t)L.W * 8, 256);
    L.hits = off;
    off = align_up(off + (size_t)L.W * 4, 256);
    L.totals_rank = off;
    off = align_up(off + (size_t)L.Gmax * 8, 256);
    L.totals_hit = off;
    off = align_up(off + (size_t)L.Gmax * 8, 256);
    L.acc = off; // cleared up to here by one memset per call
    off = align_up(off + (size_t)L.max_keys * (1 + naggs) * 8, 256);
    L.hrank = off;
    off = align_up(off + (size_t)L.W * 4, 256);
    L.cand = off;
    off = align_up(off + (size_t)L.topk_blocks * kk * sizeof(VK), 256);
    L.total = off;
    return L;
}

// Grid of a cooperative pass with `wpt` words per thread: spans of 256 x wpt
// words, at most as many blocks as are resident at once (the pass waits on a
// grid-wide barrier), each block taking `rounds` consecutive spans.  False
// when one round per block would not fit.
static bool coop_grid(const void *kern, long long W, int wpt, int Gmax, int *G, int *rounds, bool need_one_round)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GJR_THREADS, 0) != cudaSuccess || per_sm < 1)
        return false;
    const long long spans = std::max(1ll, (W + (long long)GJR_THREADS * wpt - 1) / ((long long)GJR_THREADS * wpt));
    const long long res = std::min<long long>((long long)per_sm * num_sms(), Gmax);
    if (need_one_round && spans > res)
        return false;
    *rounds = (int)((spans + res - 1) / res);
    *G = (int)((spans + *rounds - 1) / *rounds);
    return true;
}

template <int NSMAX>
static tdp_status launch_gjr_probe(const PredSet &ps, const int32_t *key, long long n, const long long *d_n,
                                   long long lo, long long D, const RankWord *bm, uint32_t *hitw, const AggSet &as,
                                   AccLayout al, long long *acc, unsigned long long *d_nmatch, int32_t *d_status,
                                   cudaStream_t s)
{
    const long long chunks = (n + GJR_CHUNK - 1) / GJR_CHUNK;
    const long long want = (chunks + GJR_PROBE_THREADS / 32 - 1) / (GJR_PROBE_THREADS / 32);
    const unsigned grid = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() * 4));
    // the staged columns: the key, then each distinct predicate column
    GJRStage sg;
    sg.n = 0;
    sg.aligned = 1;
    auto add = [&](const void *col, int size) -> int {
        for (int c = 0; c < sg.n; c++)
            if (sg.col[c] == col && sg.size[c] == size)
                return c;
        sg.col[sg.n] = col;
        sg.size[sg.n] = size;
        sg.aligned = sg.aligned && ((uintptr_t)col % 16) == 0;
        return sg.n++;
    };
    for (int c = 0; c < GJR_MAX_STAGE; c++) {
        sg.col[c] = nullptr;
        sg.size[c] = 0;
    }
    add(key, 4);
    for (int p = 0; p < TDP_MAX_PREDS; p++)
        sg.pred[p] = p < ps.n ? add(ps.col[p], dtype_size(ps.dt[p])) : 0;
    int row_bytes = 0;
    for (int c = 0; c < sg.n; c++)
        row_bytes += sg.size[c];
    // keys are int32 and [lo, hi] lies in the int32 range with D <= 2^31, so
    // (unsigned)(key - lo) < D (32-bit arithmetic) is the bounds test
    if (row_bytes <= GJR_STAGE_MAX_ROW) {
        const size_t smem = (size_t)(GJR_PROBE_THREADS / 32) * 2 * GJR_CHUNK * row_bytes;
        auto kern = gjr_probe_kernel<NSMAX>;
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GJR_PROBE_THREADS, smem) != cudaSuccess ||
            per_sm < 1)
            return TDP_ERR_CUDA;
        // persistent: one wave of resident blocks
        const unsigned g = (unsigned)std::max(1ll, std::min<long long>(want, (long long)num_sms() * per_sm));
        kern<<<g, GJR_PROBE_THREADS, smem, s>>>(ps, sg, n, d_n, (int)lo, (unsigned)D, bm, hitw, as, al, acc, d_nmatch,
                                                d_status, spin_limit());
    } else {
        gjr_probe_direct_kernel<NSMAX><<<grid, GJR_PROBE_THREADS, 0, s>>>(
            ps, key, ((uintptr_t)key % 16) == 0, n, d_n, (int)lo, (unsigned)D, bm, hitw, as, al, acc, d_nmatch);
    }
    return launch_status();
}

template <int WPT>
static tdp_status launch_gjr_hitrank(const GjrLayout &L, char *w, const uint32_t *hitw, long long cap,
                                     int64_t *d_ngroups, int32_t *d_status, int G, int rounds, cudaStream_t s)
{
    const void *kern = (const void *)gjr_hitrank_kernel<WPT>;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    unsigned *barrier = (unsigned *)&cnt[2];
    unsigned long long *totals = (unsigned long long *)(w + L.totals_hit);
    uint32_t *hrank = (uint32_t *)(w + L.hrank);
    long long W = L.W;
    long long *ng = (long long *)d_ngroups;
    const uint32_t limit = spin_limit();
    void *args[] = {(void *)&hitw, (void *)&W, (void *)&rounds, (void *)&hrank, (void *)&cap, (void *)&ng,
                    (void *)&totals, (void *)&barrier, (void *)&d_status, (void *)&limit};
    if (cudaLaunchCooperativeKernel(kern, dim3(G), dim3(GJR_THREADS), args, 0, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    return launch_status();
}

template <int NA>
static tdp_status launch_gjr_output(const GjrLayout &L, char *w, const RankWord *bm, const uint32_t *hitw,
                                    long long lo, const AggSet &as, AccLayout al, const long long *acc,
                                    int32_t *out_keys, const DenseOut &out, long long cap, cudaStream_t s)
{
    const long long warps = (L.W + 31) / 32;
    const unsigned grid = (unsigned)std::max(
        1ll, std::min<long long>((warps + GJR_THREADS / 32 - 1) / (GJR_THREADS / 32), (long long)num_sms() * 16));
    gjr_output_kernel<NA><<<grid, GJR_THREADS, 0, s>>>(bm, hitw, (const uint32_t *)(w + L.hrank), L.W, lo, as, al,
                                                       acc, out_keys, out, cap);
    return launch_status();
}

template <int WPT>
static tdp_status launch_gjr_rank(const GjrLayout &L, char *w, RankWord *bm, const AggSet &as, AccLayout al,
                                  long long *acc, int32_t *d_status, int G, int rounds, cudaStream_t s)
{
    const void *kern = (const void *)gjr_rank_kernel<WPT>;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    unsigned long long *nk = &cnt[0], *rows = &cnt[4];
    unsigned long long *totals = (unsigned long long *)(w + L.totals_rank);
    unsigned *barrier = (unsigned *)&cnt[1];
    long long W = L.W;
    const uint32_t limit = spin_limit();
    void *args[] = {(void *)&bm, (void *)&W, (void *)&rounds, (void *)&as, (void *)&al, (void *)&acc,
                    (void *)&nk, (void *)&rows, (void *)&totals, (void *)&barrier, (void *)&d_status,
                    (void *)&limit};
    if (cudaLaunchCooperativeKernel(kern, dim3(G), dim3(GJR_THREADS), args, 0, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    return launch_status();
}



// The accumulator slots of `aggs` (as make_aggset assigns them: COUNT in slot
// 0, every other aggregate in the next slot) without their columns: what the
// build and finish steps need.
static tdp_status agg_shape(const tdp_agg *aggs, int32_t naggs, AggSet *as, AccLayout *al)
{
    if (naggs < 1 || naggs > TDP_MAX_AGGS || !aggs)
        return TDP_ERR_INVALID_ARG;
    memset(as, 0, sizeof(*as));
    as->n = naggs;
    as->nslots = 1;
    al->cs = 1;
    for (int a = 0; a < naggs; a++) {
        if (aggs[a].op < TDP_AGG_COUNT || aggs[a].op > TDP_AGG_MAX)
            return TDP_ERR_INVALID_ARG;
        as->op[a] = aggs[a].op;
        as->k[a] = aggs[a].k;
        as->slot[a] = aggs[a].op == TDP_AGG_COUNT ? 0 : as->nslots++;
        if (aggs[a].op == TDP_AGG_COUNT || aggs[a].op == TDP_AGG_AVG)
            al->cs = 0;
    }
    for (int a = 0; a < naggs; a++)
        if (as->slot[a] != 0)
            as->sop[as->slot[a]] = aggs[a].op;
    al->stride = as->nslots - al->cs;
    return TDP_OK;
}

static bool gj_range_ok(int64_t key_lo, int64_t key_hi)
{
    return key_hi >= key_lo && key_hi - key_lo < (1ll << 31) && key_lo >= INT32_MIN && key_hi <= INT32_MAX;
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_groupjoin_workspace(int64_t n_build, int64_t key_lo, int64_t key_hi, int32_t naggs,
                                          int32_t topk)
{
    if (!gj_range_ok(key_lo, key_hi) || naggs < 1 || naggs > TDP_MAX_AGGS || n_build < 0 || topk < 0 ||
        topk > TK_MAXK)
        return 0;
    return gjr_layout(n_build, key_hi - key_lo + 1, naggs, topk).total;
}

extern "C" tdp_status tdp_groupjoin_build(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                                          int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild,
                                          int32_t build_key_col, int64_t key_lo, int64_t key_hi, const tdp_agg *aggs,
                                          int32_t naggs, int32_t topk, void *ws, size_t ws_bytes, int32_t *d_status,
                                          tdp_stream_t stream)
{
    if (n_build < 0 || n_build >= (1ll << 31) || !build_cols || build_key_col < 0 || build_key_col >= nbuild_cols ||
        !gj_range_ok(key_lo, key_hi) || topk < 0 || topk > TK_MAXK)
        return TDP_ERR_INVALID_ARG;
    if (build_cols[build_key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (build_cols[build_key_col].n < n_build)
        return TDP_ERR_INVALID_ARG;
    PredSet bps;
    tdp_status st = make_predset(build_cols, nbuild_cols, build_preds, nbuild_preds, n_build, &bps);
    if (st != TDP_OK)
        return st;
    AggSet as;
    AccLayout al;
    if ((st = agg_shape(aggs, naggs, &as, &al)) != TDP_OK)
        return st;
    const long long D = key_hi - key_lo + 1;
    const GjrLayout L = gjr_layout(n_build, D, naggs, topk);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws % 16) != 0)
        return TDP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    RankWord *bm = (RankWord *)(w + L.bitmap);
    long long *acc = (long long *)(w + L.acc);
    if (cudaMemsetAsync(w, 0, L.acc, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    if (n_build > 0)
        gjr_build_kernel<<<(unsigned)std::max(1ll, std::min<long long>((n_build + 256 * GJB_ROWS - 1) /
                                                                            (256 * GJB_ROWS),
                                                                        (long long)num_sms() * 6)),
                           256, 0, s>>>(
            bps, (const int32_t *)build_cols[build_key_col].data, n_build, (const long long *)d_nbuild, (int)key_lo,
            (unsigned)D, bm, &cnt[4], d_status);
    int G = 0, R = 1;
    if (coop_grid((const void *)gjr_rank_kernel<1>, L.W, 1, L.Gmax, &G, &R, true))
        return launch_gjr_rank<1>(L, w, bm, as, al, acc, d_status, G, R, s);
    if (coop_grid((const void *)gjr_rank_kernel<2>, L.W, 2, L.Gmax, &G, &R, true))
        return launch_gjr_rank<2>(L, w, bm, as, al, acc, d_status, G, R, s);
    if (coop_grid((const void *)gjr_rank_kernel<4>, L.W, 4, L.Gmax, &G, &R, false))
        return launch_gjr_rank<4>(L, w, bm, as, al, acc, d_status, G, R, s);
    return TDP_ERR_CUDA;
}

extern "C" tdp_status tdp_groupjoin_probe(const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                                          int32_t nprobe_preds, int64_t n_probe, const int64_t *d_nprobe,
                                          int32_t probe_key_col, int64_t n_build, int64_t key_lo, int64_t key_hi,
                                          const tdp_agg *aggs, int32_t naggs, int32_t topk, void *ws,
                                          size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n_probe < 0 || n_probe >= (1ll << 31) || n_build < 0 || !probe_cols || probe_key_col < 0 ||
        probe_key_col >= nprobe_cols || !gj_range_ok(key_lo, key_hi) || topk < 0 || topk > TK_MAXK)
        return TDP_ERR_INVALID_ARG;
    if (probe_cols[probe_key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (probe_cols[probe_key_col].n < n_probe)
        return TDP_ERR_INVALID_ARG;
    PredSet pps;
    tdp_status st = make_predset(probe_cols, nprobe_cols, probe_preds, nprobe_preds, n_probe, &pps);
    if (st != TDP_OK)
        return st;
    AggSet as;
    if ((st = make_aggset(probe_cols, nprobe_cols, aggs, naggs, n_probe, &as)) != TDP_OK)
        return st;
    AggSet shape;
    AccLayout al;
    if ((st = agg_shape(aggs, naggs, &shape, &al)) != TDP_OK)
        return st;
    const long long D = key_hi - key_lo + 1;
    const GjrLayout L = gjr_layout(n_build, D, naggs, topk);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (n_probe == 0)
        return TDP_OK;
    char *w = (char *)ws;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    const RankWord *bm = (const RankWord *)(w + L.bitmap);
    uint32_t *hitw = (uint32_t *)(w + L.hits);
    long long *acc = (long long *)(w + L.acc);
    const long long *dn = (const long long *)d_nprobe;
    const int32_t *pk = (const int32_t *)probe_cols[probe_key_col].data;
    cudaStream_t s = (cudaStream_t)stream;
    if (as.nslots <= 2)
        return launch_gjr_probe<2>(pps, pk, n_probe, dn, key_lo, D, bm, hitw, as, al, acc, &cnt[5], d_status, s);
    if (as.nslots <= 4)
        return launch_gjr_probe<4>(pps, pk, n_probe, dn, key_lo, D, bm, hitw, as, al, acc, &cnt[5], d_status, s);
    return launch_gjr_probe<TDP_MAX_AGGS + 1>(pps, pk, n_probe, dn, key_lo, D, bm, hitw, as, al, acc, &cnt[5],
                                              d_status, s);
}

extern "C" tdp_status tdp_groupjoin_finish(int64_t n_build, int64_t key_lo, int64_t key_hi, const tdp_agg *aggs,
                                           int32_t naggs, int32_t *out_keys, int64_t *const *out_aggs,
                                           int64_t capacity, int64_t *d_ngroups, int64_t *d_nmatch, int32_t topk,
                                           int32_t topk_agg, int64_t *out_top_vals, int32_t *out_top_keys,
                                           int64_t *d_topk, void *ws, size_t ws_bytes, int32_t *d_status,
                                           tdp_stream_t stream)
{
    if (n_build < 0 || !gj_range_ok(key_lo, key_hi) || capacity < 0 || !d_ngroups || !out_aggs ||
        (capacity > 0 && !out_keys))
        return TDP_ERR_INVALID_ARG;
    if (topk < 0 || topk > TK_MAXK ||
        (topk > 0 && (topk_agg < 0 || topk_agg >= naggs || !out_top_vals || !out_top_keys || capacity <= 0)))
        return TDP_ERR_INVALID_ARG;
    AggSet as;
    AccLayout al;
    tdp_status st = agg_shape(aggs, naggs, &as, &al);
    if (st != TDP_OK)
        return st;
    for (int a = 0; a < naggs; a++)
        if (capacity > 0 && !out_aggs[a])
            return TDP_ERR_INVALID_ARG;
    const long long D = key_hi - key_lo + 1;
    const GjrLayout L = gjr_layout(n_build, D, naggs, topk);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    const RankWord *bm = (const RankWord *)(w + L.bitmap);
    const uint32_t *hitw = (const uint32_t *)(w + L.hits);
    const long long *acc = (const long long *)(w + L.acc);
    if (d_nmatch && cudaMemcpyAsync(d_nmatch, &cnt[5], sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    DenseOut out;
    for (int k = 0; k < TDP_MAX_KEYS; k++) {
        out.key_out[k] = nullptr;
        out.key_dt[k] = TDP_I32;
    }
    for (int a = 0; a < TDP_MAX_AGGS; a++)
        out.agg_out[a] = a < naggs ? (long long *)out_aggs[a] : nullptr;
    {
        int G = 0, R = 1;
        if (coop_grid((const void *)gjr_hitrank_kernel<1>, L.W, 1, L.Gmax, &G, &R, true))
            st = launch_gjr_hitrank<1>(L, w, hitw, capacity, d_ngroups, d_status, G, R, s);
        else if (coop_grid((const void *)gjr_hitrank_kernel<2>, L.W, 2, L.Gmax, &G, &R, true))
            st = launch_gjr_hitrank<2>(L, w, hitw, capacity, d_ngroups, d_status, G, R, s);
        else if (coop_grid((const void *)gjr_hitrank_kernel<4>, L.W, 4, L.Gmax, &G, &R, false))
            st = launch_gjr_hitrank<4>(L, w, hitw, capacity, d_ngroups, d_status, G, R, s);
        else
            st = TDP_ERR_CUDA;
        if (st != TDP_OK)
            return st;
    }
    if (naggs == 1)
        st = launch_gjr_output<1>(L, w, bm, hitw, key_lo, as, al, acc, out_keys, out, capacity, s);
    else if (naggs == 2)
        st = launch_gjr_output<2>(L, w, bm, hitw, key_lo, as, al, acc, out_keys, out, capacity, s);
    else if (naggs <= 4)
        st = launch_gjr_output<4>(L, w, bm, hitw, key_lo, as, al, acc, out_keys, out, capacity, s);
    else
        st = launch_gjr_output<TDP_MAX_AGGS>(L, w, bm, hitw, key_lo, as, al, acc, out_keys, out, capacity, s);
    if (st != TDP_OK)
        return st;
    if (topk > 0) {
        VK *cand = (VK *)(w + L.cand);
        gjr_topk_blocks_kernel<<<L.topk_blocks, GJR_THREADS, 0, s>>>((const long long *)out_aggs[topk_agg], out_keys,
                                                                    (const long long *)d_ngroups, capacity, topk,
                                                                    cand, &cnt[3]);
        gjr_topk_final_kernel<<<1, GJR_THREADS, 0, s>>>(cand, (long long)L.topk_blocks * topk, topk, &cnt[3],
                                                       (const long long *)d_ngroups, capacity,
                                                       (long long *)out_top_vals, out_top_keys, (long long *)d_topk);
    }
    return launch_status();
}

extern "C" tdp_status tdp_groupjoin(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                                    int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild,
                                    int32_t build_key_col, const tdp_col *probe_cols, int32_t nprobe_cols,
                                    const tdp_pred *probe_preds, int32_t nprobe_preds, int64_t n_probe,
                                    const int64_t *d_nprobe, int32_t probe_key_col, int64_t key_lo, int64_t key_hi,
                                    const tdp_agg *aggs, int32_t naggs, int32_t *out_keys, int64_t *const *out_aggs,
                                    int64_t capacity, int64_t *d_ngroups, int64_t *d_nmatch, int32_t topk,
                                    int32_t topk_agg, int64_t *out_top_vals, int32_t *out_top_keys, int64_t *d_topk,
                                    void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    // every argument is checked before anything is launched
    if (!probe_cols || probe_key_col < 0 || probe_key_col >= nprobe_cols || n_probe < 0 || n_probe >= (1ll << 31) ||
        capacity < 0 || !d_ngroups || !out_aggs || (capacity > 0 && !out_keys) || topk < 0 || topk > TK_MAXK ||
        (topk > 0 && (topk_agg < 0 || topk_agg >= naggs || !out_top_vals || !out_top_keys || capacity <= 0)))
        return TDP_ERR_INVALID_ARG;
    if (probe_cols[probe_key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    {
        PredSet pps;
        AggSet as;
        tdp_status st = make_predset(probe_cols, nprobe_cols, probe_preds, nprobe_preds, n_probe, &pps);
        if (st == TDP_OK)
            st = make_aggset(probe_cols, nprobe_cols, aggs, naggs, n_probe, &as);
        if (st != TDP_OK)
            return st;
        if (probe_cols[probe_key_col].n < n_probe)
            return TDP_ERR_INVALID_ARG;
        for (int a = 0; a < naggs; a++)
            if (capacity > 0 && !out_aggs[a])
                return TDP_ERR_INVALID_ARG;
    }
    tdp_status st = tdp_groupjoin_build(build_cols, nbuild_cols, build_preds, nbuild_preds, n_build, d_nbuild,
                                        build_key_col, key_lo, key_hi, aggs, naggs, topk, ws, ws_bytes, d_status,
                                        stream);
    if (st != TDP_OK)
        return st;
    st = tdp_groupjoin_probe(probe_cols, nprobe_cols, probe_preds, nprobe_preds, n_probe, d_nprobe, probe_key_col,
                             n_build, key_lo, key_hi, aggs, naggs, topk, ws, ws_bytes, d_status, stream);
    if (st != TDP_OK)
        return st;
    return tdp_groupjoin_finish(n_build, key_lo, key_hi, aggs, naggs, out_keys, out_aggs, capacity, d_ngroups,
                                d_nmatch, topk, topk_agg, out_top_vals, out_top_keys, d_topk, ws, ws_bytes, d_status,
                                stream);
}
