// K7: group-join where the group key is the join key, over a rank code of
// the build keys.
//
// SELECT k, aggs(probe columns) FROM build JOIN probe ON build.key = probe.key
// WHERE build preds AND probe preds GROUP BY k ORDER BY k, for unique build
// keys bounded by [lo, hi] (the column metadata of Sec. 2 that selects an
// operator strategy).  Sec. 2 (Data Encoding) keeps an order-preserving
// dictionary code per column; here the build side's key set is turned into
// exactly such a code on the device, and the code is the accumulator index:
//
//   1. build: every qualifying build row sets bit (key - lo) of a bitmap of
//      D = hi - lo + 1 bits, stored as words of 32 keys with a rank field
//      beside each word ({bits, rank}: 8 bytes per 32 keys, 3.75 MB for
//      D = 15M).  A bit that is already set is a duplicate build key.
//   2. rank: an exclusive scan of the words' popcounts (decoupled look-back
//      over tiles of 1024 words) writes each word's rank; the code of key k
//      is then rank[w] + popc(bits[w] below k's bit), a dense number in
//      0..B-1 in ascending key order (B build keys).  The same pass sets the
//      B accumulator rows to their initial values.
//   3. probe: persistent blocks stream tiles of the probe key and predicate
//      columns through two shared-memory buffers filled by bulk copies;
//      every qualifying row looks its key up in the bitmap (one 8-byte load,
//      L2-resident), and a hit gathers the row's aggregate inputs and adds
//      them into accumulator row `code` with 64-bit atomics (L2-resident:
//      B x slots x 8 bytes).
//   4. finalize: tiles of 1024 bitmap words; every set bit whose accumulator
//      row counted a match is one output group.  Walking the bits in order
//      walks the keys in order, so the groups come out sorted with no sort;
//      the key is lo + 32 w + bit.  Output offsets by decoupled look-back.
//
// Nothing is written per match and no partition or sort of the matches is
// needed; the only per-row traffic is the probe-side columns.
#include <algorithm>

#include "groupby.cuh"

namespace tdp {

constexpr int GJR_THREADS = 256;
constexpr int GJR_WORDS = GJR_THREADS * 4; // bitmap words per scan / finalize tile
constexpr int GJR_MAX_RPT = 16;            // probe rows per thread per tile (fewer for wide rows)
constexpr int GJR_MAX_STAGE = 1 + TDP_MAX_PREDS;

struct __align__(8) RankWord {
    uint32_t bits;
    uint32_t rank;
};

// ---------------------------------------------------------------- 1. build

__global__ void gjr_build_kernel(PredSet ps, const int32_t *__restrict__ key, long long n, const long long *d_n,
                                 long long lo, long long D, RankWord *bm, int32_t *d_status)
{
    if (d_n)
        n = min(*d_n, n);
    const long long r0 = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r0 >= n)
        return;
    const unsigned m = eval_preds4(ps, r0, n);
    if (!m)
        return;
    int k[4];
    if (r0 + 3 < n && ((uintptr_t)key % 16) == 0) {
        const int4 kk = __ldg((const int4 *)(key + r0));
        k[0] = kk.x, k[1] = kk.y, k[2] = kk.z, k[3] = kk.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++)
            k[e] = (m >> e & 1) ? key[r0 + e] : 0;
    }
    int err = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        if (!(m >> e & 1))
            continue;
        const long long d = (long long)k[e] - lo;
        if (d < 0 || d >= D) { // a build key outside its declared bounds
            err |= TDP_ERR_OVERFLOW;
            continue;
        }
        const uint32_t bit = 1u << (d & 31);
        const uint32_t old = atomicOr(&bm[d >> 5].bits, bit);
        if (old & bit)
            err |= TDP_ERR_DUP_BUILD_KEY;
    }
    if (err)
        set_status(d_status, err);
}

// ----------------------------------------------------------------- 2. rank

// Exclusive block scan of one unsigned per thread; returns the thread's
// exclusive prefix and (in *total) the block total.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *s_warp, unsigned *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    unsigned before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < GJR_THREADS / 32; w++) {
        const unsigned t = s_warp[w];
        before += w < warp ? t : 0;
        all += t;
    }
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(GJR_THREADS) gjr_rank_kernel(RankWord *bm, long long W, AggSet as,
                                                               long long *acc, unsigned long long *d_nkeys,
                                                               long long *d_nmatch, unsigned long long *tile_status,
                                                               unsigned *ticket, int32_t *d_status, uint32_t limit,
                                                               long long ntiles)
{
    __shared__ long long s_tile;
    __shared__ unsigned s_warp[GJR_THREADS / 32];
    __shared__ unsigned long long s_excl;
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    if (threadIdx.x <= TDP_MAX_AGGS)
        s_init[threadIdx.x] = slot_init(as, threadIdx.x);
    __syncthreads();
    const long long tile = s_tile;
    if (tile == 0 && threadIdx.x == 0 && d_nmatch)
        *d_nmatch = 0; // the probe, which runs after this kernel, adds its matches
    const long long w0 = tile * GJR_WORDS + 4ll * threadIdx.x;
    uint32_t b[4];
#pragma unroll
    for (int j = 0; j < 4; j++)
        b[j] = w0 + j < W ? bm[w0 + j].bits : 0u;
    const unsigned c = __popc(b[0]) + __popc(b[1]) + __popc(b[2]) + __popc(b[3]);
    unsigned total;
    const unsigned pre = block_excl_scan(c, s_warp, &total);
    if (threadIdx.x < 32) {
        const unsigned long long e = lookback_exclusive(tile_status, tile, total, limit, d_status);
        if (threadIdx.x == 0) {
            s_excl = e;
            if (tile == ntiles - 1)
                *d_nkeys = e + total;
        }
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
    unsigned r = (unsigned)(excl + pre);
#pragma unroll
    for (int j = 0; j < 4; j++)
        if (w0 + j < W) {
            bm[w0 + j].rank = r;
            r += __popc(b[j]);
        }
    // initial values of this tile's accumulator rows (contiguous codes)
    const int NS = as.nslots;
    long long *a0 = acc + (long long)excl * NS;
    for (long long i = threadIdx.x; i < (long long)total * NS; i += GJR_THREADS)
        a0[i] = s_init[i % NS];
}

// ---------------------------------------------------------------- 3. probe

// Columns a probe tile stages in shared memory: the key and the predicate
// columns, each once.
struct GJRStage {
    const void *col[GJR_MAX_STAGE];
    int32_t size[GJR_MAX_STAGE];
    int32_t n;
    int32_t aligned;           // every staged column 16-byte aligned
    int32_t pred[TDP_MAX_PREDS]; // stage index of predicate p's column
};

__device__ __forceinline__ long long staged_val(const unsigned char *col, int dt, int li)
{
    switch (dt) {
    case TDP_I8: return ((const int8_t *)col)[li];
    case TDP_U8: return ((const uint8_t *)col)[li];
    case TDP_I32: return ((const int32_t *)col)[li];
    default: return ((const long long *)col)[li];
    }
}

// Aggregate input of slot s for probe row `row`, read from global memory
// (read once: evict-first in L2).
__device__ __forceinline__ long long gather_int(const void *p, int dt, long long row, uint64_t pol)
{
    switch (dt) {
    case TDP_I8: return ((const int8_t *)p)[row];
    case TDP_U8: return ((const uint8_t *)p)[row];
    case TDP_I32: return ldg_hint((const int32_t *)p + row, pol);
    default: return ldg_hint((const long long *)p + row, pol);
    }
}

// NSMAX: accumulator slots the kernel is compiled for (COUNT + sums);
// BATCH: lookups in flight per thread (fewer when more values are gathered).
template <int NSMAX, int BATCH>
__global__ void __launch_bounds__(GJR_THREADS, 3)
    gjr_probe_kernel(PredSet ps, GJRStage sg, int rpt, long long n_host, const long long *d_n, long long lo,
                     long long D, const RankWord *bm, AggSet as, long long *acc, unsigned long long *d_nmatch,
                     int32_t *d_status, uint32_t limit)
{
    const int T = GJR_THREADS * rpt;
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    extern __shared__ __align__(128) unsigned char gjr_smem[];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    __shared__ uint32_t s_off[GJR_MAX_STAGE];
    const int tid = threadIdx.x;
    const int NS = as.nslots;
    if (tid <= TDP_MAX_AGGS)
        s_ops[tid] = slot_op(as, tid);
    uint32_t row_bytes = 0;
    for (int c = 0; c < sg.n; c++)
        row_bytes += sg.size[c];
    if (tid == 0) {
        uint32_t off = 0;
        for (int c = 0; c < sg.n; c++) {
            s_off[c] = off;
            off += T * sg.size[c];
        }
        mbar_init(&s_full[0], 1);
        mbar_init(&s_full[1], 1);
    }
    __syncthreads();
    const uint64_t stream_pol = l2_evict_first(), table_pol = l2_evict_last();
    const long long ntiles = (n + T - 1) / T;
    auto bulk_ok = [&](long long t) { return sg.aligned && (t + 1) * T <= n; };
    auto issue = [&](long long t, int b) {
        unsigned char *buf = gjr_smem + (size_t)b * T * row_bytes;
        mbar_arrive_expect_tx(&s_full[b], T * row_bytes);
        for (int c = 0; c < sg.n; c++)
            bulk_load_hint(buf + s_off[c], (const char *)sg.col[c] + (size_t)t * T * sg.size[c], T * sg.size[c],
                           &s_full[b], stream_pol);
    };
    if (tid == 0 && blockIdx.x < ntiles && bulk_ok(blockIdx.x))
        issue(blockIdx.x, 0);
    __syncthreads();

    bool late = false;
    unsigned long long matches = 0;
    uint32_t phase = 0; // bit b: parity of buffer b's next phase
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int b = it & 1;
        unsigned char *buf = gjr_smem + (size_t)b * T * row_bytes;
        const long long tn = t + gridDim.x;
        if (tid == 0 && tn < ntiles && bulk_ok(tn))
            issue(tn, b ^ 1); // that buffer was released at the end of the previous tile
        if (bulk_ok(t)) {
            late |= !mbar_wait(&s_full[b], (phase >> b) & 1u, limit);
            phase ^= 1u << b;
        } else {
            for (int li = tid; li < T; li += GJR_THREADS) {
                const long long idx = t * T + li;
                if (idx >= n)
                    break;
                for (int c = 0; c < sg.n; c++) {
                    unsigned char *d = buf + s_off[c];
                    switch (sg.size[c]) {
                    case 8: ((long long *)d)[li] = ((const long long *)sg.col[c])[idx]; break;
                    case 4: ((int32_t *)d)[li] = ((const int32_t *)sg.col[c])[idx]; break;
                    default: d[li] = ((const uint8_t *)sg.col[c])[idx]; break;
                    }
                }
            }
            __syncthreads();
        }
        const int32_t *skey = (const int32_t *)(buf + s_off[0]);
#pragma unroll 1
        for (int h = 0; h < rpt; h += BATCH) {
            // (a) predicates and the bitmap word of every qualifying key
            RankWord w[BATCH];
            int bitpos[BATCH];
#pragma unroll
            for (int r = 0; r < BATCH; r++) {
                bitpos[r] = -1;
                const int li = tid + (h + r) * GJR_THREADS;
                if (h + r >= rpt || t * T + li >= n)
                    continue;
                bool q = true;
                for (int p = 0; p < ps.n; p++) {
                    const long long v = staged_val(buf + s_off[sg.pred[p]], ps.dt[p], li);
                    q = q && range_holds64(v, ps.lo[p], (unsigned long long)(ps.hi[p] - ps.lo[p]), (unsigned)ps.neg[p]);
                }
                const long long d = (long long)skey[li] - lo;
                if (q && d >= 0 && d < D) {
                    const unsigned long long u = ldg_hint((const unsigned long long *)(bm + (d >> 5)), table_pol);
                    w[r].bits = (uint32_t)u;
                    w[r].rank = (uint32_t)(u >> 32);
                    bitpos[r] = (int)(d & 31);
                }
            }
            // (b) hits: code, then the aggregate inputs of all hits in flight
            uint32_t code[BATCH];
            long long va[BATCH][NSMAX], vb[BATCH][NSMAX];
#pragma unroll
            for (int r = 0; r < BATCH; r++) {
                code[r] = 0xffffffffu;
                if (bitpos[r] < 0 || !((w[r].bits >> bitpos[r]) & 1u))
                    continue;
                code[r] = w[r].rank + __popc(w[r].bits & ((1u << bitpos[r]) - 1u));
                const long long row = t * T + tid + (h + r) * GJR_THREADS;
#pragma unroll
                for (int s = 1; s < NSMAX; s++) {
                    if (s >= NS)
                        break;
                    va[r][s] = gather_int(as.sa[s], as.sadt[s], row, stream_pol);
                    vb[r][s] = as.sop[s] == TDP_AGG_SUM_MUL_KMINUS ? gather_int(as.sb[s], as.sbdt[s], row, stream_pol)
                                                                    : 0;
                }
            }
            // (c) accumulate (atomics without a return value)
#pragma unroll
            for (int r = 0; r < BATCH; r++) {
                if (code[r] == 0xffffffffu)
                    continue;
                matches++;
                long long *dst = acc + (long long)code[r] * NS;
                atomicAdd((unsigned long long *)dst, 1ull);
#pragma unroll
                for (int s = 1; s < NSMAX; s++) {
                    if (s >= NS)
                        break;
                    long long v = va[r][s];
                    if (as.sop[s] == TDP_AGG_SUM_MUL_KMINUS)
                        v *= as.sk[s] - vb[r][s];
                    acc_update(dst + s, s_ops[s], v);
                }
            }
        }
        __syncthreads(); // buffer b free for the tile after next
    }
    if (late)
        set_status(d_status, TDP_ERR_TIMEOUT);
    // match count: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        matches += __shfl_xor_sync(0xffffffffu, matches, o);
    if ((tid & 31) == 0 && matches && d_nmatch)
        atomicAdd(d_nmatch, matches);
}

// ------------------------------------------------------------- 4. finalize

__global__ void __launch_bounds__(GJR_THREADS) gjr_finalize_kernel(const RankWord *bm, long long W, long long lo,
                                                                   AggSet as, const long long *acc,
                                                                   int32_t *out_keys, DenseOut out, long long cap,
                                                                   long long *d_ngroups,
                                                                   unsigned long long *tile_status, unsigned *ticket,
                                                                   int32_t *d_status, uint32_t limit,
                                                                   long long ntiles)
{
    __shared__ long long s_tile;
    __shared__ unsigned s_warp[GJR_THREADS / 32];
    __shared__ unsigned long long s_excl;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const int NS = as.nslots;
    const long long w0 = tile * GJR_WORDS + 4ll * threadIdx.x;
    // matched keys of the thread's 4 words: bit j of hit[i] = key 32 (w0+i) + j
    uint32_t hit[4];
    uint32_t rank0 = 0;
    unsigned c = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        hit[i] = 0;
        if (w0 + i >= W)
            continue;
        const RankWord e = bm[w0 + i];
        if (i == 0)
            rank0 = e.rank;
        uint32_t bits = e.bits;
        uint32_t code = e.rank;
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            if (acc[(long long)code * NS] > 0)
                hit[i] |= 1u << j;
            code++;
        }
        c += __popc(hit[i]);
    }
    unsigned total;
    const unsigned pre = block_excl_scan(c, s_warp, &total);
    if (threadIdx.x < 32) {
        const unsigned long long e = lookback_exclusive(tile_status, tile, total, limit, d_status);
        if (threadIdx.x == 0) {
            s_excl = e;
            if (tile == ntiles - 1) {
                *d_ngroups = (long long)(e + total);
                if ((long long)(e + total) > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    long long pos = (long long)s_excl + pre;
    uint32_t code = rank0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (w0 + i >= W)
            break;
        const uint32_t bits = bm[w0 + i].bits;
        uint32_t all = bits;
        while (all) {
            const int j = __ffs(all) - 1;
            all &= all - 1;
            if ((hit[i] >> j) & 1u) {
                if (pos < cap) {
                    out_keys[pos] = (int32_t)(lo + 32 * (w0 + i) + j);
                    for (int a = 0; a < as.n; a++)
                        out.agg_out[a][pos] = agg_final(as, a, acc + (long long)code * NS);
                }
                pos++;
            }
            code++;
        }
    }
}

// ----------------------------------------------------------------- host

struct GjrLayout {
    size_t counters, bitmap, scan_status, fin_status, acc, total;
    long long W, scan_tiles, max_keys;
};

static GjrLayout gjr_layout(long long n_build, long long D, int naggs)
{
    GjrLayout L;
    L.W = (D + 31) / 32;
    L.scan_tiles = (L.W + GJR_WORDS - 1) / GJR_WORDS;
    L.max_keys = std::max(0ll, std::min(n_build, D));
    size_t off = 0;
    L.counters = off; // [0] build keys, [1] scan ticket, [2] finalize ticket
    off += 256;
    L.bitmap = off;
    off = align_up(off + (size_t)L.W * 8, 256);
    L.scan_status = off;
    off = align_up(off + (size_t)L.scan_tiles * 8, 256);
    L.fin_status = off;
    off = align_up(off + (size_t)L.scan_tiles * 8, 256);
    L.acc = off; // cleared up to here by one memset per call
    off = align_up(off + (size_t)L.max_keys * (1 + naggs) * 8, 256);
    L.total = off;
    return L;
}

template <int NSMAX, int BATCH>
static tdp_status launch_gjr_probe(const PredSet &ps, const GJRStage &sg, long long n, const long long *d_n,
                                   long long lo, long long D, const RankWord *bm, const AggSet &as, long long *acc,
                                   unsigned long long *d_nmatch, int32_t *d_status, cudaStream_t s)
{
    size_t row_bytes = 0;
    for (int c = 0; c < sg.n; c++)
        row_bytes += sg.size[c];
    // two tile buffers within 200 KiB
    int rpt = GJR_MAX_RPT;
    while (rpt > 1 && 2 * (size_t)GJR_THREADS * rpt * row_bytes > 200 * 1024)
        rpt >>= 1;
    const long long T = (long long)GJR_THREADS * rpt;
    const size_t smem = 2 * (size_t)T * row_bytes;
    auto kern = gjr_probe_kernel<NSMAX, BATCH>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    const int per_sm = std::max(1, std::min(3, (int)((220 * 1024) / (smem + 1024))));
    const long long tiles = (n + T - 1) / T;
    const unsigned grid = (unsigned)std::max(1ll, std::min<long long>(tiles, (long long)num_sms() * per_sm));
    kern<<<grid, GJR_THREADS, smem, s>>>(ps, sg, rpt, n, d_n, lo, D, bm, as, acc, d_nmatch, d_status, spin_limit());
    return launch_status();
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_groupjoin_workspace(int64_t n_build, int64_t key_lo, int64_t key_hi, int32_t naggs)
{
    if (key_hi < key_lo || key_hi - key_lo >= (1ll << 31) || naggs < 1 || naggs > TDP_MAX_AGGS || n_build < 0)
        return 0;
    return gjr_layout(n_build, key_hi - key_lo + 1, naggs).total;
}

extern "C" tdp_status tdp_groupjoin(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                                    int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild,
                                    int32_t build_key_col, const tdp_col *probe_cols, int32_t nprobe_cols,
                                    const tdp_pred *probe_preds, int32_t nprobe_preds, int64_t n_probe,
                                    const int64_t *d_nprobe, int32_t probe_key_col, int64_t key_lo, int64_t key_hi,
                                    const tdp_agg *aggs, int32_t naggs, int32_t *out_keys, int64_t *const *out_aggs,
                                    int64_t capacity, int64_t *d_ngroups, int64_t *d_nmatch, void *ws,
                                    size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n_build < 0 || n_build >= (1ll << 31) || n_probe < 0 || n_probe >= (1ll << 31) || !build_cols ||
        !probe_cols || build_key_col < 0 || build_key_col >= nbuild_cols || probe_key_col < 0 ||
        probe_key_col >= nprobe_cols || key_hi < key_lo || key_hi - key_lo >= (1ll << 31) || capacity < 0 ||
        !d_ngroups || !out_aggs || (capacity > 0 && !out_keys))
        return TDP_ERR_INVALID_ARG;
    if (build_cols[build_key_col].dtype != TDP_I32 || probe_cols[probe_key_col].dtype != TDP_I32)
        return TDP_ERR_UNSUPPORTED_DTYPE;
    if (build_cols[build_key_col].n < n_build || probe_cols[probe_key_col].n < n_probe)
        return TDP_ERR_INVALID_ARG;
    PredSet bps, pps;
    tdp_status st = make_predset(build_cols, nbuild_cols, build_preds, nbuild_preds, n_build, &bps);
    if (st != TDP_OK)
        return st;
    if ((st = make_predset(probe_cols, nprobe_cols, probe_preds, nprobe_preds, n_probe, &pps)) != TDP_OK)
        return st;
    AggSet as;
    if ((st = make_aggset(probe_cols, nprobe_cols, aggs, naggs, n_probe, &as)) != TDP_OK)
        return st;
    for (int a = 0; a < naggs; a++)
        if (capacity > 0 && !out_aggs[a])
            return TDP_ERR_INVALID_ARG;
    const long long D = key_hi - key_lo + 1;
    const GjrLayout L = gjr_layout(n_build, D, naggs);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws % 16) != 0)
        return TDP_ERR_INVALID_ARG;
    // the staged probe columns: the key, then each distinct predicate column
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
    add(probe_cols[probe_key_col].data, 4);
    for (int p = 0; p < TDP_MAX_PREDS; p++)
        sg.pred[p] = p < pps.n ? add(pps.col[p], dtype_size(pps.dt[p])) : 0;

    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    unsigned long long *cnt = (unsigned long long *)(w + L.counters);
    RankWord *bm = (RankWord *)(w + L.bitmap);
    long long *acc = (long long *)(w + L.acc);
    if (cudaMemsetAsync(w, 0, L.acc, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    if (n_build > 0)
        gjr_build_kernel<<<(unsigned)((n_build + 1023) / 1024), 256, 0, s>>>(
            bps, (const int32_t *)build_cols[build_key_col].data, n_build, (const long long *)d_nbuild, key_lo, D,
            bm, d_status);
    gjr_rank_kernel<<<(unsigned)L.scan_tiles, GJR_THREADS, 0, s>>>(
        bm, L.W, as, acc, &cnt[0], (long long *)d_nmatch, (unsigned long long *)(w + L.scan_status),
        (unsigned *)&cnt[1], d_status, spin_limit(), L.scan_tiles);
    if ((st = launch_status()) != TDP_OK)
        return st;
    if (n_probe > 0) {
        const long long *dn = (const long long *)d_nprobe;
        unsigned long long *nm = (unsigned long long *)d_nmatch;
        if (as.nslots <= 2)
            st = launch_gjr_probe<2, 8>(pps, sg, n_probe, dn, key_lo, D, bm, as, acc, nm, d_status, s);
        else if (as.nslots <= 4)
            st = launch_gjr_probe<4, 4>(pps, sg, n_probe, dn, key_lo, D, bm, as, acc, nm, d_status, s);
        else
            st = launch_gjr_probe<TDP_MAX_AGGS + 1, 2>(pps, sg, n_probe, dn, key_lo, D, bm, as, acc, nm, d_status,
                                                       s);
        if (st != TDP_OK)
            return st;
    }
    DenseOut out;
    for (int k = 0; k < TDP_MAX_KEYS; k++) {
        out.key_out[k] = nullptr;
        out.key_dt[k] = TDP_I32;
    }
    for (int a = 0; a < TDP_MAX_AGGS; a++)
        out.agg_out[a] = a < naggs ? (long long *)out_aggs[a] : nullptr;
    gjr_finalize_kernel<<<(unsigned)L.scan_tiles, GJR_THREADS, 0, s>>>(
        bm, L.W, key_lo, as, acc, out_keys, out, capacity, (long long *)d_ngroups,
        (unsigned long long *)(w + L.fin_status), (unsigned *)&cnt[2], d_status, spin_limit(), L.scan_tiles);
    return launch_status();
}
