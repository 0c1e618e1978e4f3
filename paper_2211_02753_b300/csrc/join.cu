// K6/K7: open-addressing hash equi-join (build, probe, fused probe+group-by).
//
// Table (the caller's nslots x 8 bytes, nslots a power of two >= 8, base
// 32-byte aligned): nslots slots of (int32 key, int32 payload), in buckets
// of 4 slots -- 32 bytes, one DRAM/L2 sector, one vector load that brings a
// bucket's keys and their payloads together.  A key hashes (multiplicative,
// Fibonacci) to a bucket; a bucket that is full and does not hold the key
// passes the search on to the next bucket (linear probing over buckets).  An
// empty slot holds (INT32_MIN, 0), so INT32_MIN cannot be stored (the build
// flags it as TDP_ERR_OVERFLOW).  Insert: one load of the bucket, a 64-bit
// CAS of key and payload into its first empty slot (on a lost race the CAS
// result tells whether the winner holds the same key: a duplicate).
// Lookup: one 32-byte load of the bucket nearly always decides it, payload
// included.  At the default load factor (<= 1/2) a lookup crosses into a
// second bucket for a few percent of the keys; the walk is bounded by
// min(nbuckets, 8192) buckets, beyond which TDP_ERR_CAPACITY is reported.
// (With the keys and the payloads in two arrays, a lookup that wanted the
// payload made two sector requests; the join chain's probe + aggregate ran
// 1.5x longer so.)
//
// Probe (compaction in probe order): one tile of T = 256 x 4 x STEPS probe
// rows per block, tiles in block order:
//   1. the tile of every predicate column and of the key column goes to
//      shared memory (one bulk copy per column for a full aligned tile of a
//      plain scan, evict-first in L2; plain loads otherwise);
//   2. predicate mask of lane rows lrow + j*128 + 0..3 (step j);
//   3. the tile-local indices of qualifying rows form a dense queue (ballot
//      ranks); every thread resolves queue entries tid, tid + 256, ... eight
//      at a time (eight bucket loads in flight, table loads evict-last in L2)
//      and marks found rows in a byte flag per row; found payloads overwrite
//      their keys in shared memory when the caller wants payloads;
//   4. ballots over the flags rank the hits; their tile-local indices are
//      staged at their ranks while warp 0 runs the decoupled look-back for
//      the tile's output offset;
//   5. coalesced output: probe row, payload, gathered columns.
//
// Probe + aggregate: the build payload is the group key (dense range
// [lo, hi]).  Persistent blocks take tiles of probe rows in grid-stride
// order, the staged columns of the next tile arriving by bulk copy while the
// current one is processed; matched rows are added into a per-block
// shared-memory cache of 2048 groups (open addressing on the group id, two
// probes), which absorbs Zipf-hot groups; groups that find no cache slot go
// straight to the global dense accumulator table with 64-bit atomics (a
// short probe sequence: once the cache is full, the cold half of a Zipf
// stream misses, and a miss should cost two shared reads, not eight).  Cache contents are merged into the
// global table at the end, then the non-empty groups are compacted in order.
#include <algorithm>

#include "coop.cuh"
#include "filter_api.cuh"
#include "groupby.cuh"
#include "radix.cuh"

namespace tdp {

constexpr uint32_t EMPTY_KEY = 0x80000000u; // INT32_MIN
constexpr int BUCKET = 4;                   // (key, payload) slots per bucket: 32 bytes, one sector
constexpr unsigned long long MAX_BUCKETS = 1ull << 13;
// an empty slot: key INT32_MIN, payload 0 (as one little-endian 64-bit word)
constexpr unsigned long long EMPTY_SLOT = (unsigned long long)EMPTY_KEY;

struct TableView {
    const uint32_t *w; // slot i: key w[2i], payload w[2i + 1]; bucket b: slots 4b .. 4b+3
    unsigned bmask;    // nbuckets - 1
    int lgb;           // log2(nbuckets)
    unsigned steps;    // bucket walk bound
};

__device__ __forceinline__ unsigned bucket_of(int key, int lgb)
{
    return lgb == 0 ? 0u : ((unsigned)key * 0x9E3779B1u) >> (32 - lgb);
}

struct Oct {
    uint32_t v[8];
};

// 32-byte read-only load with an L2 policy: a bucket's four (key, payload)
// slots.
__device__ __forceinline__ Oct load_oct(const uint32_t *p, uint64_t pol)
{
    Oct r;
    asm("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
          "=r"(r.v[7])
        : "l"(p), "l"(pol));
    return r;
}

// The bucket b of the table (its first word).
__device__ __forceinline__ const uint32_t *bucket_ptr(const TableView &tv, unsigned b)
{
    return tv.w + (size_t)b * (2 * BUCKET);
}

// Position of the first slot holding `key` (0..3) in a loaded bucket, -1 if
// an empty slot comes first (the key is absent), -2 if the bucket is full of
// other keys (the walk goes on).  Slots fill in order and are never freed,
// so no empty slot precedes a stored key.
__device__ __forceinline__ int scan_bucket(const Oct &k, uint32_t key)
{
    int res = -2;
#pragma unroll
    for (int i = BUCKET - 1; i >= 0; i--) {
        if (k.v[2 * i] == key)
            res = i;
        else if (k.v[2 * i] == EMPTY_KEY)
            res = -1;
    }
    return res;
}

// The payload of slot i (0..3) of a loaded bucket.
__device__ __forceinline__ int32_t pick(const Oct &p, int i)
{
    int32_t r = 0;
#pragma unroll
    for (int j = 0; j < BUCKET; j++)
        r = j == i ? (int32_t)p.v[2 * j + 1] : r;
    return r;
}

// The payload of slot `slot` of the table.
__device__ __forceinline__ int32_t tv_pay(const TableView &tv, long long slot)
{
    return (int32_t)__ldg(tv.w + 2 * slot + 1);
}

// Continues a lookup whose first bucket b0 was full of other keys: walks the
// following buckets.  Returns the slot of the key (>= 0), -1 if absent, -2
// past the walk bound.
__device__ __noinline__ long long lookup_tail(const uint32_t *w, unsigned bmask, unsigned steps, uint32_t key,
                                              unsigned b0, uint64_t pol)
{
    unsigned b = b0;
    for (unsigned s = 1; s < steps; s++) {
        b = (b + 1) & bmask;
        // two 16-byte loads here: ptxas of CUDA 13.0 fails on a 32-byte load
        // inside a non-inlined function
        const uint32_t *bk = w + (size_t)b * (2 * BUCKET);
        Oct k;
        asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
            : "=r"(k.v[0]), "=r"(k.v[1]), "=r"(k.v[2]), "=r"(k.v[3])
            : "l"(bk), "l"(pol));
        asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
            : "=r"(k.v[4]), "=r"(k.v[5]), "=r"(k.v[6]), "=r"(k.v[7])
            : "l"(bk + 4), "l"(pol));
        const int r = scan_bucket(k, key);
        if (r >= 0)
            return (long long)b * BUCKET + r;
        if (r == -1)
            return -1;
    }
    return -2;
}

// Every slot empty: (INT32_MIN, 0), two slots per 16-byte store.
__global__ void fill_empty_kernel(uint32_t *w, long long nslots)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 e = make_uint4(EMPTY_KEY, 0u, EMPTY_KEY, 0u);
    for (; i < nslots / 2; i += (long long)gridDim.x * blockDim.x)
        ((uint4 *)w)[i] = e;
}

__global__ void join_build_kernel(PredSet ps, const int32_t *__restrict__ key, const int32_t *__restrict__ payload,
                                  long long n, const long long *d_n, uint32_t *tw, int lgb,
                                  unsigned steps, int32_t *d_status)
{
    if (d_n)
        n = min(*d_n, n);
    const unsigned bmask = (1u << lgb) - 1;
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
    int p[4];
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
            p[e] = (m >> e & 1) && payload ? payload[r0 + e] : 0;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
        if (!(m >> e & 1))
            continue;
        const uint32_t kv = (uint32_t)k[e];
        const int pv = payload ? p[e] : (int)(r0 + e);
        if (kv == EMPTY_KEY) {
            err |= TDP_ERR_OVERFLOW;
            continue;
        }
        unsigned b = bucket_of(k[e], lgb);
        bool done = false;
        for (unsigned s = 0; s < steps && !done; s++, b = (b + 1) & bmask) {
            uint32_t *bk = tw + (size_t)b * (2 * BUCKET);
            const uint4 lo = __ldcg((const uint4 *)bk), hi = __ldcg((const uint4 *)bk + 1);
            const uint32_t cur[BUCKET] = {lo.x, lo.z, hi.x, hi.z}; // the slots' keys
            // slots are visited in order; a slot passed over holds another key
            // for good (no deletes), so two inserts of one key meet on one slot
#pragma unroll
            for (int i = 0; i < BUCKET; i++) {
                if (done)
                    break;
                uint32_t c = cur[i];
                if (c == EMPTY_KEY) {
                    // key and payload claimed together: one 64-bit CAS of the slot
                    const unsigned long long got = atomicCAS(
                        (unsigned long long *)(bk + 2 * i), EMPTY_SLOT,
                        ((unsigned long long)(uint32_t)pv << 32) | kv);
                    c = (uint32_t)got;
                    if (got == EMPTY_SLOT) {
                        done = true;
                        break;
                    }
                }
                if (c == kv) {
                    err |= TDP_ERR_DUP_BUILD_KEY;
                    done = true;
                }
            }
        }
        if (!done)
            err |= TDP_ERR_CAPACITY;
    }
    if (err)
        set_status(d_status, err);
}

constexpr int JP_THREADS = 256;
constexpr int JP_BATCH = 5;     // key-bucket lookups in flight per thread
constexpr int JP_BATCH_PAY = 3; // with their payload buckets

template <int STEPS, bool PAY>
__global__ void __launch_bounds__(JP_THREADS, 3) join_probe_kernel(
    TableView tv, PredSet ps, const int32_t *__restrict__ key, bool key_vec, long long n, const int32_t *sel,
    const long long *d_nsel, int32_t *out_row, int32_t *out_payload, GatherSet gs, long long cap, long long *d_count,
    unsigned long long *tile_status, int32_t *d_status, uint32_t limit, long long num_tiles)
{
    constexpr int T = JP_THREADS * 4 * STEPS;
    extern __shared__ __align__(128) unsigned char jp_smem[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned s_warp[JP_THREADS / 32];
    __shared__ unsigned long long s_excl;

    const long long tile = blockIdx.x;
    const long long m = d_nsel ? min(*d_nsel, n) : n;
    const long long ibase = tile * T;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lrow = warp * (STEPS * 128) + 4 * lane;
    uint32_t pbytes = 0;
    for (int p = 0; p < ps.n; p++)
        pbytes += T * (uint32_t)dtype_size_dev(ps.dt[p]);
    const uint32_t kofs = max(pbytes, (uint32_t)T * 4);
    int32_t *sk = (int32_t *)(jp_smem + kofs);              // keys, then payloads in place
    uint16_t *queue = (uint16_t *)jp_smem;                  // after the predicates: qualifying rows
    unsigned char *found = jp_smem + 2 * T;                 // one flag byte per row
    int32_t *stage = (int32_t *)jp_smem;                    // finally: the hits in output order
    const uint64_t stream_pol = l2_evict_first(), table_pol = l2_evict_last();

    // 1. stage the tile
    bool bulk = !sel && key_vec && ibase + T <= m;
    for (int p = 0; p < ps.n; p++)
        bulk = bulk && ps.vec_ok[p];
    if (bulk) {
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            mbar_arrive_expect_tx(&s_bar, pbytes + T * 4);
            uint32_t off = 0;
            for (int p = 0; p < ps.n; p++) {
                const int sz = dtype_size_dev(ps.dt[p]);
                bulk_load_hint(jp_smem + off, (const char *)ps.col[p] + (size_t)ibase * sz, T * sz, &s_bar,
                               stream_pol);
                off += T * sz;
            }
            bulk_load_hint(sk, key + ibase, T * 4, &s_bar, stream_pol);
        }
    } else {
        for (int i = tid; i < T; i += JP_THREADS) {
            const long long idx = ibase + i;
            if (idx >= m)
                continue;
            const long long row = sel ? sel[idx] : idx;
            sk[i] = key[row];
            uint32_t off = 0;
            for (int p = 0; p < ps.n; p++) {
                const int sz = dtype_size_dev(ps.dt[p]);
                const long long v = load_int(ps.col[p], ps.dt[p], row);
                unsigned char *d = jp_smem + off + (size_t)i * sz;
                if (sz == 8)
                    *(long long *)d = v;
                else if (sz == 4)
                    *(int32_t *)d = (int32_t)v;
                else
                    *d = (unsigned char)v;
                off += T * sz;
            }
        }
    }
    __syncthreads();
    if (bulk && !mbar_wait(&s_bar, 0, limit))
        set_status(d_status, TDP_ERR_TIMEOUT);

    // 2. predicate mask (rows past the end are never set)
    unsigned msk[STEPS];
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        const long long r = ibase + lrow + j * 128;
        msk[j] = r + 3 < m ? 0xfu : (r + 2 < m ? 0x7u : (r + 1 < m ? 0x3u : (r < m ? 0x1u : 0u)));
    }
    {
        uint32_t off = 0;
        for (int p = 0; p < ps.n; p++) {
            pred_test_smem<STEPS>(ps, p, jp_smem + off, lrow, msk);
            off += T * dtype_size_dev(ps.dt[p]);
        }
    }

    // 3. queue of qualifying rows, then lookups
    const unsigned lt = lanemask_lt();
    unsigned rank[STEPS], wtot = 0;
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        unsigned cnt = 0, pre = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const unsigned b = __ballot_sync(0xffffffffu, (msk[j] >> e) & 1u);
            cnt += __popc(b);
            pre += __popc(b & lt);
        }
        rank[j] = cnt << 16 | pre;
        wtot += cnt;
    }
    if (lane == 0)
        s_warp[warp] = wtot;
    __syncthreads(); // predicate tiles consumed
    unsigned qoff = 0, qtot = 0;
#pragma unroll
    for (int w = 0; w < JP_THREADS / 32; w++) {
        const unsigned t = s_warp[w];
        qoff += w < warp ? t : 0;
        qtot += t;
    }
    {
        unsigned pos = qoff;
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            unsigned q = pos + (rank[j] & 0xffffu);
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (msk[j] >> e & 1)
                    queue[q++] = (uint16_t)(lrow + j * 128 + e);
            pos += rank[j] >> 16;
        }
        for (int i = tid; i < T / 4; i += JP_THREADS)
            ((uint32_t *)found)[i] = 0u;
    }
    __syncthreads();
    constexpr bool want_pay = PAY;
    // 8 registers per key bucket in flight, 16 with its payload bucket
    constexpr int NB = PAY ? JP_BATCH_PAY : JP_BATCH;
    bool gave_up = false;
    for (unsigned base = 0; base < qtot; base += JP_THREADS * NB) {
        int li[NB];
        uint32_t kq[NB];
        int pv[NB];
        long long slot[NB]; // slot of the found key, -1 if absent
        Oct wk[NB]; // the buckets: keys and payloads
#pragma unroll
        for (int k = 0; k < NB; k++) {
            const unsigned q = base + tid + k * JP_THREADS;
            li[k] = q < qtot ? queue[q] : -1;
            kq[k] = li[k] >= 0 ? (uint32_t)sk[li[k]] : EMPTY_KEY;
            if (kq[k] != EMPTY_KEY)
                wk[k] = load_oct(bucket_ptr(tv, bucket_of((int)kq[k], tv.lgb)), table_pol);
        }
#pragma unroll
        for (int k = 0; k < NB; k++) {
            slot[k] = -1;
            pv[k] = 0;
            if (kq[k] == EMPTY_KEY)
                continue;
            const unsigned b = bucket_of((int)kq[k], tv.lgb);
            const int r = scan_bucket(wk[k], kq[k]);
            if (r >= 0) {
                slot[k] = (long long)b * BUCKET + r;
                if constexpr (PAY)
                    pv[k] = pick(wk[k], r);
            } else if (r == -2) {
                const long long t = lookup_tail(tv.w, tv.bmask, tv.steps, kq[k], b, table_pol);
                gave_up |= t == -2;
                if (t >= 0) {
                    slot[k] = t;
                    if constexpr (PAY)
                        pv[k] = tv_pay(tv, t);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NB; k++)
            if (slot[k] >= 0) {
                found[li[k]] = 1;
                if (want_pay)
                    sk[li[k]] = pv[k];
            }
    }
    if (gave_up)
        set_status(d_status, TDP_ERR_CAPACITY);
    __syncthreads();

    // 4. ranks of the hits; staged tile-local indices; look-back
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        const uint32_t f = *(const uint32_t *)(found + lrow + j * 128);
        msk[j] = (f & 1u) | (f >> 7 & 2u) | (f >> 14 & 4u) | (f >> 21 & 8u);
    }
    unsigned btot = 0, woff = 0;
    wtot = 0;
#pragma unroll
    for (int j = 0; j < STEPS; j++) {
        unsigned cnt = 0, pre = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const unsigned b = __ballot_sync(0xffffffffu, (msk[j] >> e) & 1u);
            cnt += __popc(b);
            pre += __popc(b & lt);
        }
        rank[j] = cnt << 16 | pre;
        wtot += cnt;
    }
    if (lane == 0)
        s_warp[warp] = wtot;
    __syncthreads(); // queue and flags consumed
#pragma unroll
    for (int w = 0; w < JP_THREADS / 32; w++) {
        const unsigned t = s_warp[w];
        woff += w < warp ? t : 0;
        btot += t;
    }
    {
        unsigned pos = woff;
#pragma unroll
        for (int j = 0; j < STEPS; j++) {
            unsigned q = pos + (rank[j] & 0xffffu);
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (msk[j] >> e & 1)
                    stage[q++] = lrow + j * 128 + e;
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

    // 5. output
    const long long excl = (long long)s_excl;
    const unsigned lim = (unsigned)max(0ll, min((long long)btot, cap - excl));
    if (out_row || out_payload)
        for (unsigned i = tid; i < lim; i += JP_THREADS) {
            const int l = stage[i];
            if (out_row)
                out_row[excl + i] = sel ? sel[ibase + l] : (int32_t)(ibase + l);
            if (out_payload)
                out_payload[excl + i] = sk[l];
        }
    for (int g = 0; g < gs.n; g++) {
        const void *col = gs.col[g];
        void *out = gs.out[g];
        if (col == (const void *)key && !PAY) { // the probe key is still in shared memory
            for (unsigned i = tid; i < lim; i += JP_THREADS)
                ((int32_t *)out)[excl + i] = sk[stage[i]];
            continue;
        }
        switch (gs.size[g]) {
        case 8:
#pragma unroll 4
            for (unsigned i = tid; i < lim; i += JP_THREADS) {
                const long long row = sel ? sel[ibase + stage[i]] : ibase + stage[i];
                ((long long *)out)[excl + i] = ldg_hint((const long long *)col + row, stream_pol);
            }
            break;
        case 4:
#pragma unroll 4
            for (unsigned i = tid; i < lim; i += JP_THREADS) {
                const long long row = sel ? sel[ibase + stage[i]] : ibase + stage[i];
                ((int32_t *)out)[excl + i] = ldg_hint((const int32_t *)col + row, stream_pol);
            }
            break;
        case 2:
            for (unsigned i = tid; i < lim; i += JP_THREADS) {
                const long long row = sel ? sel[ibase + stage[i]] : ibase + stage[i];
                ((uint16_t *)out)[excl + i] = ((const uint16_t *)col)[row];
            }
            break;
        default:
            for (unsigned i = tid; i < lim; i += JP_THREADS) {
                const long long row = sel ? sel[ibase + stage[i]] : ibase + stage[i];
                ((uint8_t *)out)[excl + i] = ((const uint8_t *)col)[row];
            }
            break;
        }
    }
}

// ------------------------------------------------------- probe + aggregate

constexpr int GJ_CACHE = 2048;
constexpr int GJ_PROBES = 2;
constexpr int GJ_MAX_STAGE = 16; // distinct columns staged per tile

// The columns a group-join tile stages in shared memory (key, predicate and
// aggregate columns, each once), and where every use finds its column.
struct GJStage {
    const void *col[GJ_MAX_STAGE];
    int32_t size[GJ_MAX_STAGE];
    int32_t n;
    int32_t aligned;                 // every staged column 16-byte aligned
    int32_t key;                     // stage index of the probe key
    int32_t pred[TDP_MAX_PREDS];     // stage index of predicate p's column
    int32_t sa[TDP_MAX_AGGS + 1];    // stage index of slot s's a column (-1: none)
    int32_t sb[TDP_MAX_AGGS + 1];    // and of its b column
};

__device__ __forceinline__ long long stage_val(const unsigned char *col, int size, int dt, int li)
{
    switch (dt) {
    case TDP_I8: return ((const int8_t *)col)[li];
    case TDP_U8: return ((const uint8_t *)col)[li];
    case TDP_I32: return ((const int32_t *)col)[li];
    default: return size == 8 ? ((const long long *)col)[li] : ((const int32_t *)col)[li];
    }
}

// Finds (or claims) the cache entry of group gid; nullptr when the probe
// sequence of the cache is full.
__device__ __forceinline__ long long *gj_cache_slot(unsigned *s_key, long long *s_acc, int NS, long long gid)
{
    const unsigned tag = (unsigned)gid + 1u;
    unsigned h = ((unsigned)gid * 0x9E3779B1u) >> 21; // 11 bits: GJ_CACHE = 2048
    for (int q = 0; q < GJ_PROBES; q++) {
        unsigned cur = s_key[h];
        if (cur == 0)
            cur = atomicCAS(&s_key[h], 0u, tag);
        if (cur == 0 || cur == tag)
            return s_acc + h * NS;
        h = (h + 1) & (GJ_CACHE - 1);
    }
    return nullptr;
}

// Persistent group-join: tiles of T = 256 x RPT probe rows in grid-stride
// order.  Thread 0 bulk-copies the staged columns of the block's next tile
// into the other of two shared buffers while the block works on the current
// one (a ragged or unaligned tile is loaded by all threads instead).  Row
// li = tid + k*256 of the tile (k < RPT) is looked up in batches of 4: the
// first half of its key bucket and of its payload bucket are loaded
// together, so one round trip resolves keys in the first four slots; the
// second half, and then the following buckets, are read only when needed.
template <int RPT>
__global__ void __launch_bounds__(JP_THREADS, 3) join_probe_agg_kernel(TableView tv, PredSet ps, GJStage sg,
                                                                       long long n_host, const long long *d_n,
                                                                       long long lo, long long D, AggSet as,
                                                                       long long *gacc, int32_t *d_status,
                                                                       uint32_t limit)
{
    constexpr int T = JP_THREADS * RPT;
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    extern __shared__ __align__(128) long long gj_smem[];
    const int NS = as.nslots;
    long long *s_acc = gj_smem;                                   // [GJ_CACHE][NS]
    unsigned *s_key = (unsigned *)(gj_smem + GJ_CACHE * NS);      // [GJ_CACHE], gid + 1, 0 = empty
    unsigned char *bufs = (unsigned char *)(s_key + GJ_CACHE);    // 2 x T x row bytes
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ int s_ops[TDP_MAX_AGGS + 1];
    __shared__ long long s_init[TDP_MAX_AGGS + 1];
    __shared__ uint32_t s_off[GJ_MAX_STAGE];
    const int tid = threadIdx.x;
    if (tid <= TDP_MAX_AGGS) {
        int sl = tid, op = TDP_AGG_SUM;
        for (int a = 0; a < as.n; a++)
            if (as.slot[a] == sl && sl != 0)
                op = as.op[a];
        s_ops[sl] = op;
        s_init[sl] = slot_init(as, sl);
    }
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
    for (int e = tid; e < GJ_CACHE; e += JP_THREADS) {
        s_key[e] = 0;
        for (int sl = 0; sl < NS; sl++)
            s_acc[e * NS + sl] = s_init[sl];
    }
    const uint64_t stream_pol = l2_evict_first(), table_pol = l2_evict_last();
    const long long ntiles = (n + T - 1) / T;
    auto bulk_ok = [&](long long t) { return sg.aligned && (t + 1) * T <= n; };
    auto issue = [&](long long t, int b) {
        unsigned char *buf = bufs + (size_t)b * T * row_bytes;
        mbar_arrive_expect_tx(&s_full[b], T * row_bytes);
        for (int c = 0; c < sg.n; c++)
            bulk_load_hint(buf + s_off[c], (const char *)sg.col[c] + (size_t)t * T * sg.size[c], T * sg.size[c],
                           &s_full[b], stream_pol);
    };
    if (tid == 0 && blockIdx.x < ntiles && bulk_ok(blockIdx.x))
        issue(blockIdx.x, 0);
    __syncthreads();

    bool bad = false, gave_up = false, late = false;
    uint32_t phase = 0; // bit b: parity of buffer b's next phase
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int b = it & 1;
        unsigned char *buf = bufs + (size_t)b * T * row_bytes;
        const long long tn = t + gridDim.x;
        if (tid == 0 && tn < ntiles && bulk_ok(tn))
            issue(tn, b ^ 1); // that buffer was released at the end of the previous tile
        if (bulk_ok(t)) {
            late |= !mbar_wait(&s_full[b], (phase >> b) & 1u, limit);
            phase ^= 1u << b;
        } else {
            for (int li = tid; li < T; li += JP_THREADS) {
                const long long idx = t * T + li;
                if (idx >= n)
                    break;
                for (int c = 0; c < sg.n; c++) {
                    unsigned char *d = buf + s_off[c];
                    switch (sg.size[c]) {
                    case 8: ((long long *)d)[li] = ((const long long *)sg.col[c])[idx]; break;
                    case 4: ((int32_t *)d)[li] = ((const int32_t *)sg.col[c])[idx]; break;
                    case 2: ((uint16_t *)d)[li] = ((const uint16_t *)sg.col[c])[idx]; break;
                    default: d[li] = ((const uint8_t *)sg.col[c])[idx]; break;
                    }
                }
            }
            __syncthreads();
        }
        const int32_t *skey = (const int32_t *)(buf + s_off[sg.key]);
#pragma unroll
        for (int h = 0; h < RPT; h += 4) {
            // predicates, then one round trip for 4 buckets (a bucket is one
            // sector of four (key, payload) slots)
            uint32_t kq[4];
            Oct wk[4];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                kq[r] = EMPTY_KEY;
                if (h + r >= RPT)
                    continue;
                const int li = tid + (h + r) * JP_THREADS;
                if (t * T + li >= n)
                    continue;
                bool q = true;
                for (int p = 0; p < ps.n; p++) {
                    const int c = sg.pred[p];
                    const long long v = stage_val(buf + s_off[c], sg.size[c], ps.dt[p], li);
                    q = q && range_holds64(v, ps.lo[p], (unsigned long long)(ps.hi[p] - ps.lo[p]),
                                           (unsigned)ps.neg[p]);
                }
                if (q)
                    kq[r] = (uint32_t)skey[li];
                if (kq[r] != EMPTY_KEY)
                    wk[r] = load_oct(bucket_ptr(tv, bucket_of((int)kq[r], tv.lgb)), table_pol);
            }
#pragma unroll
            for (int r = 0; r < 4; r++) {
                if (kq[r] == EMPTY_KEY)
                    continue;
                const int li = tid + (h + r) * JP_THREADS;
                const unsigned bk = bucket_of((int)kq[r], tv.lgb);
                int pos = scan_bucket(wk[r], kq[r]);
                int32_t pay = pos >= 0 ? pick(wk[r], pos) : 0;
                if (pos == -2) { // bucket full of other keys: the walk
                    const long long slot = lookup_tail(tv.w, tv.bmask, tv.steps, kq[r], bk, table_pol);
                    gave_up |= slot == -2;
                    if (slot < 0)
                        continue;
                    pay = tv_pay(tv, slot);
                } else if (pos < 0) {
                    continue;
                }
                // aggregate the row into its group
                const long long gid = (long long)pay - lo;
                if (gid < 0 || gid >= D) {
                    bad = true;
                    continue;
                }
                long long *dst = gj_cache_slot(s_key, s_acc, NS, gid);
                if (!dst)
                    dst = gacc + gid * NS;
                atomicAdd((unsigned long long *)&dst[0], 1ull);
                for (int sl = 1; sl < NS; sl++) {
                    long long va = stage_val(buf + s_off[sg.sa[sl]], sg.size[sg.sa[sl]], as.sadt[sl], li);
                    if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                        va *= as.sk[sl] - stage_val(buf + s_off[sg.sb[sl]], sg.size[sg.sb[sl]], as.sbdt[sl], li);
                    acc_update(&dst[sl], s_ops[sl], va);
                }
            }
        }
        __syncthreads(); // buffer b free for the tile after next
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
    if (gave_up)
        set_status(d_status, TDP_ERR_CAPACITY);
    if (late)
        set_status(d_status, TDP_ERR_TIMEOUT);
    __syncthreads();
    for (int e = tid; e < GJ_CACHE; e += JP_THREADS) {
        const unsigned tag = s_key[e];
        if (!tag)
            continue;
        const long long gid = (long long)tag - 1;
        for (int sl = 0; sl < NS; sl++) {
            const long long v = s_acc[e * NS + sl];
            if (v != s_init[sl])
                acc_update(&gacc[gid * NS + sl], s_ops[sl], v);
        }
    }
}

static int log2_of(long long x)
{
    int lg = 0;
    while ((1ll << lg) < x)
        lg++;
    return lg;
}

// nslots: a power of two in [8, 2^32]; the table 32-byte aligned (one
// bucket per sector)
static bool table_ok(const void *table, long long nslots)
{
    return nslots >= 8 && nslots <= (1ll << 32) && (nslots & (nslots - 1)) == 0 && ((uintptr_t)table % 32) == 0;
}

static TableView table_view(const uint64_t *table, long long nslots)
{
    TableView tv;
    tv.w = (const uint32_t *)table;
    const long long nb = nslots / BUCKET;
    tv.lgb = log2_of(nb);
    tv.bmask = (unsigned)(nb - 1);
    tv.steps = (unsigned)std::min<unsigned long long>((unsigned long long)nb, MAX_BUCKETS);
    return tv;
}

// Rows per probe tile: shared memory max(P, 4T) + 4T <= 64 KiB, P = T x the
// predicate bytes of a row.
static int probe_steps(const PredSet &ps)
{
    int row_bytes = 0;
    for (int p = 0; p < ps.n; p++)
        row_bytes += dtype_size(ps.dt[p]);
    int steps = 8;
    while (steps > 1 && (size_t)JP_THREADS * 4 * steps * (std::max(row_bytes, 4) + 4) > 64 * 1024)
        steps >>= 1;
    return steps;
}

template <int STEPS>
static tdp_status launch_probe(const TableView &tv, const PredSet &ps, const int32_t *key, long long n,
                               const int32_t *sel, const long long *d_nsel, int32_t *out_row, int32_t *out_payload,
                               const GatherSet &gs, long long cap, long long *d_count, void *ws, int32_t *d_status,
                               cudaStream_t s)
{
    constexpr long long T = JP_THREADS * 4 * STEPS;
    const long long tiles = (n + T - 1) / T;
    size_t pbytes = 0;
    for (int p = 0; p < ps.n; p++)
        pbytes += (size_t)T * dtype_size(ps.dt[p]);
    const size_t smem = std::max(pbytes, (size_t)T * 4) + (size_t)T * 4;
    auto kern = out_payload ? join_probe_kernel<STEPS, true> : join_probe_kernel<STEPS, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    unsigned long long *status = (unsigned long long *)((char *)ws + 16);
    cudaMemsetAsync(status, 0, (size_t)tiles * 8, s);
    kern<<<(unsigned)tiles, JP_THREADS, smem, s>>>(tv, ps, key, ((uintptr_t)key % 16) == 0, n, sel, d_nsel, out_row,
                                                    out_payload, gs, cap, d_count, status, d_status, spin_limit(),
                                                    tiles);
    return launch_status();
}

// The staged-column plan of a group-join: each distinct column once.
static bool make_gjstage(const PredSet &ps, const AggSet &as, const void *key, GJStage *sg)
{
    sg->n = 0;
    sg->aligned = 1;
    auto add = [&](const void *col, int size) -> int {
        for (int c = 0; c < sg->n; c++)
            if (sg->col[c] == col && sg->size[c] == size)
                return c;
        if (sg->n == GJ_MAX_STAGE)
            return -1;
        sg->col[sg->n] = col;
        sg->size[sg->n] = size;
        sg->aligned = sg->aligned && ((uintptr_t)col % 16) == 0;
        return sg->n++;
    };
    for (int c = 0; c < GJ_MAX_STAGE; c++) {
        sg->col[c] = nullptr;
        sg->size[c] = 0;
    }
    if ((sg->key = add(key, 4)) < 0)
        return false;
    for (int p = 0; p < TDP_MAX_PREDS; p++) {
        sg->pred[p] = -1;
        if (p < ps.n && (sg->pred[p] = add(ps.col[p], dtype_size(ps.dt[p]))) < 0)
            return false;
    }
    for (int sl = 0; sl <= TDP_MAX_AGGS; sl++) {
        sg->sa[sl] = sg->sb[sl] = -1;
        if (sl == 0 || sl >= as.nslots)
            continue;
        if ((sg->sa[sl] = add(as.sa[sl], dtype_size(as.sadt[sl]))) < 0)
            return false;
        if (as.sop[sl] == TDP_AGG_SUM_MUL_KMINUS && (sg->sb[sl] = add(as.sb[sl], dtype_size(as.sbdt[sl]))) < 0)
            return false;
    }
    return true;
}

template <int RPT>
static tdp_status launch_gj(const TableView &tv, const PredSet &ps, const GJStage &sg, const AggSet &as, long long n,
                            const long long *d_n, long long lo, long long D, long long *acc, int32_t *d_status,
                            cudaStream_t s, size_t row_bytes)
{
    constexpr long long T = JP_THREADS * RPT;
    const size_t smem = (size_t)GJ_CACHE * as.nslots * 8 + GJ_CACHE * 4 + 2 * T * row_bytes;
    auto kern = join_probe_agg_kernel<RPT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TDP_ERR_CUDA;
    const int per_sm = std::max(1, std::min(3, (int)((220 * 1024) / (smem + 1024))));
    const long long tiles = (n + T - 1) / T;
    const unsigned grid = (unsigned)std::max(1ll, std::min<long long>(tiles, (long long)num_sms() * per_sm));
    kern<<<grid, JP_THREADS, smem, s>>>(tv, ps, sg, n, d_n, lo, D, as, acc, d_status, spin_limit());
    return launch_status();
}

// Rows per thread of a group-join tile (at most 4, so that three blocks, and
// three group caches, fit on an SM): two tile buffers within 64 KiB.
static tdp_status launch_probe_agg(const TableView &tv, const PredSet &ps, const GJStage &sg, const AggSet &as,
                                   long long n, const long long *d_n, long long lo, long long D, long long *acc,
                                   int32_t *d_status, cudaStream_t s)
{
    size_t row_bytes = 0;
    for (int c = 0; c < sg.n; c++)
        row_bytes += sg.size[c];
    int rpt = 4;
    while (rpt > 1 && 2 * (size_t)JP_THREADS * rpt * row_bytes > 64 * 1024)
        rpt >>= 1;
    switch (rpt) {
    case 4: return launch_gj<4>(tv, ps, sg, as, n, d_n, lo, D, acc, d_status, s, row_bytes);
    case 2: return launch_gj<2>(tv, ps, sg, as, n, d_n, lo, D, acc, d_status, s, row_bytes);
    default: return launch_gj<1>(tv, ps, sg, as, n, d_n, lo, D, acc, d_status, s, row_bytes);
    }
}

// ----------------------------------------------------------- N:M join
//
// Inner equi-join with repeated build keys: every (probe row, build row)
// pair with equal keys, in probe-row order and, for one probe row, in
// build-row order.
//   1. the build side's qualifying rows and their keys (the filter kernel,
//      fused gather), the keys made unsigned order-preserving (sign bit
//      flipped) and sorted with their row ids (onesweep radix sort, stable:
//      equal keys keep build-row order);
//   2. the runs of equal keys (cooperative pass): the distinct keys in order
//      and the start of each run (CSR offsets, one more than the runs);
//   3. the distinct keys into the open-addressing table with their run
//      number as payload (tdp_join_build, unique keys);
//   4. probe (cooperative): every qualifying probe row looks its key up once
//      (four rows a thread in flight) and keeps the run number; the run
//      lengths give each block its output offset; then each span of 2048
//      probe rows writes its pairs as one contiguous range, the block's
//      threads taking consecutive outputs (an output finds its probe row by
//      binary search over the rows' offsets in shared memory), so the writes
//      coalesce whatever the run lengths.

constexpr int NM_IPT = 8; // elements per thread per span of the cooperative passes

__global__ void nm_pack_kernel(const int32_t *key, long long n_max, const long long *d_n, uint32_t *ukey)
{
    const long long n = min(*d_n, n_max);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ukey[i] = (uint32_t)key[i] ^ 0x80000000u;
}

// Runs of equal keys in the sorted keys skey[0..nb): dkey[u] the u-th
// distinct key (signed), start[u] its first position; start[U] = nb, *d_runs
// = U.
__global__ void __launch_bounds__(COOP_THREADS) nm_runs_kernel(const uint32_t *skey, long long nb_max,
                                                               const long long *d_nb, int rounds, int32_t *dkey,
                                                               int32_t *start, long long *d_runs,
                                                               unsigned long long *totals, unsigned *barrier,
                                                               int32_t *d_status, uint32_t limit)
{
    __shared__ unsigned long long s_red[COOP_THREADS / 32];
    __shared__ unsigned s_warp[COOP_THREADS / 32];
    const long long nb = min(*d_nb, nb_max);
    const long long span = (long long)COOP_THREADS * NM_IPT;
    const long long b0 = (long long)blockIdx.x * rounds * span;
    auto head = [&](long long i) { return i < nb && (i == 0 || skey[i] != skey[i - 1]); };
    unsigned long long c = 0;
    for (int r = 0; r < rounds; r++) {
        const long long i0 = b0 + r * span + (long long)threadIdx.x * NM_IPT;
#pragma unroll
        for (int e = 0; e < NM_IPT; e++)
            c += head(i0 + e);
    }
    const unsigned long long total = block_sum(c, s_red);
    unsigned long long run = coop_block_prefix(total, s_red, totals, barrier, limit, d_status);
    for (int r = 0; r < rounds; r++) {
        const long long i0 = b0 + r * span + (long long)threadIdx.x * NM_IPT;
        unsigned h = 0;
#pragma unroll
        for (int e = 0; e < NM_IPT; e++)
            h |= head(i0 + e) ? 1u << e : 0u;
        unsigned tot;
        long long u = (long long)run + block_excl_scan(__popc(h), s_warp, &tot);
#pragma unroll
        for (int e = 0; e < NM_IPT; e++)
            if (h >> e & 1u) {
                dkey[u] = (int32_t)(skey[i0 + e] ^ 0x80000000u);
                start[u] = (int32_t)(i0 + e);
                u++;
            }
        run += tot;
        __syncthreads(); // s_warp reused by the next span's scan
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        start[run] = (int32_t)nb;
        *d_runs = (long long)run;
    }
}

__global__ void __launch_bounds__(COOP_THREADS) nm_probe_kernel(
    TableView tv, PredSet ps, const int32_t *__restrict__ key, long long n_host, const long long *d_n, int rounds,
    const int32_t *start, const uint32_t *srow, int32_t *pord, int32_t *out_probe, int32_t *out_build, long long cap,
    long long *d_count, unsigned long long *totals, unsigned *barrier, int32_t *d_status, uint32_t limit)
{
    __shared__ unsigned long long s_red[COOP_THREADS / 32];
    __shared__ unsigned long long s_warp[COOP_THREADS / 32];
    const long long n = d_n ? min(*d_n, n_host) : n_host;
    const long long span = (long long)COOP_THREADS * NM_IPT;
    const long long b0 = (long long)blockIdx.x * rounds * span;
    const uint64_t pol = l2_evict_last();
    bool gave_up = false;
    // 1. one lookup per qualifying row; the run number is kept per row
    unsigned long long c = 0;
    for (int r = 0; r < rounds; r++) {
        const long long i0 = b0 + r * span + (long long)threadIdx.x * NM_IPT;
        if (i0 >= n)
            continue;
        unsigned m = 0;
        for (int q = 0; q < NM_IPT; q += 4)
            m |= eval_preds4(ps, i0 + q, n) << q;
        // four rows at a time, in stages (their buckets, then their
        // payloads, then their run lengths), so that the rows' loads overlap
#pragma unroll
        for (int e0 = 0; e0 < NM_IPT; e0 += 4) {
            uint32_t kq[4];
            Oct kb[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const long long i = i0 + e0 + e;
                kq[e] = (i < n && (m >> (e0 + e) & 1u)) ? (uint32_t)key[i] : EMPTY_KEY;
                if (kq[e] != EMPTY_KEY)
                    kb[e] = load_oct(bucket_ptr(tv, bucket_of((int)kq[e], tv.lgb)), pol);
            }
            int u[4]; // the run number (the payload), -1: no match
            long long tail[4]; // a walked lookup's slot (its payload read below)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                u[e] = -1;
                tail[e] = -1;
                if (kq[e] == EMPTY_KEY)
                    continue;
                const unsigned b = bucket_of((int)kq[e], tv.lgb);
                const int r = scan_bucket(kb[e], kq[e]);
                if (r >= 0) {
                    u[e] = pick(kb[e], r);
                } else if (r == -2) {
                    tail[e] = lookup_tail(tv.w, tv.bmask, tv.steps, kq[e], b, pol);
                    gave_up |= tail[e] == -2;
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (tail[e] >= 0)
                    u[e] = tv_pay(tv, tail[e]);
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (u[e] >= 0)
                    c += (unsigned long long)(start[u[e] + 1] - start[u[e]]);
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (i0 + e0 + e < n)
                    pord[i0 + e0 + e] = u[e];
        }
    }
    if (gave_up)
        set_status(d_status, TDP_ERR_CAPACITY);
    const unsigned long long total = block_sum(c, s_red);
    unsigned long long run = coop_block_prefix(total, s_red, totals, barrier, limit, d_status);
    // 2. every matching probe row writes its run of build rows at its offset.
    // A span's pairs are one contiguous range of the output; the block writes
    // it together: output k of the span finds its row q (the last whose
    // offset is <= k) by binary search over the rows' offsets in shared
    // memory, so consecutive threads write consecutive pairs.
    __shared__ unsigned long long s_roff[COOP_THREADS * NM_IPT + 1];
    __shared__ int32_t s_base[COOP_THREADS * NM_IPT]; // the row's run starts at srow[s_base]
    constexpr int SR = COOP_THREADS * NM_IPT;
    for (int r = 0; r < rounds; r++) {
        const long long i0 = b0 + r * span + (long long)threadIdx.x * NM_IPT;
        int u[NM_IPT], s0[NM_IPT];
        unsigned long long len[NM_IPT], cr = 0;
#pragma unroll
        for (int e = 0; e < NM_IPT; e++)
            u[e] = i0 + e < n ? pord[i0 + e] : -1;
#pragma unroll
        for (int e = 0; e < NM_IPT; e++) {
            s0[e] = u[e] >= 0 ? start[u[e]] : 0;
            len[e] = u[e] >= 0 ? (unsigned long long)(start[u[e] + 1] - s0[e]) : 0ull;
            cr += len[e];
        }
        unsigned long long tot;
        unsigned long long off = block_excl_scan64(cr, s_warp, &tot);
#pragma unroll
        for (int e = 0; e < NM_IPT; e++) {
            s_roff[threadIdx.x * NM_IPT + e] = off;
            s_base[threadIdx.x * NM_IPT + e] = s0[e];
            off += len[e];
        }
        if (threadIdx.x == 0)
            s_roff[SR] = tot;
        __syncthreads();
        const long long rbase = b0 + r * span; // probe row of span row 0
        static_assert((SR & (SR - 1)) == 0, "span rows: a power of two");
        // four outputs a thread at a time (their searches and gathers overlap)
        for (unsigned long long k0 = threadIdx.x; k0 < tot; k0 += 4 * COOP_THREADS) {
            int lo[4] = {0, 0, 0, 0}; // the last row whose offset is <= k (s_roff[0] = 0)
#pragma unroll
            for (int st = SR / 2; st > 0; st >>= 1)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (s_roff[lo[j] + st] <= k0 + j * COOP_THREADS)
                        lo[j] += st;
            uint32_t b[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const unsigned long long k = k0 + j * COOP_THREADS;
                b[j] = k < tot ? srow[s_base[lo[j]] + (long long)(k - s_roff[lo[j]])] : 0u;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const unsigned long long k = k0 + j * COOP_THREADS;
                const long long pos = (long long)(run + k);
                if (k < tot && pos < cap) {
                    out_probe[pos] = (int32_t)(rbase + lo[j]);
                    out_build[pos] = (int32_t)b[j];
                }
            }
        }
        run += tot;
        __syncthreads(); // s_warp, s_roff, s_base reused by the next span
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *d_count = (long long)run;
        if ((long long)run > cap)
            set_status(d_status, TDP_ERR_CAPACITY);
    }
}

struct NmLayout {
    size_t counters, filter_ws, brow, bkey, ukey, skey, srow, radix, dkey, start, table, pord, totals, total;
    long long nslots;
    int Gmax;
};

static NmLayout nm_layout(long long n_build, long long n_probe)
{
    NmLayout L;
    const long long nb = std::max(1ll, n_build);
    L.nslots = tdp_join_default_slots(nb);
    L.Gmax = 8 * num_sms();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.counters = take(256); // [0] build rows kept, [1] runs, [2] barrier (runs), [3] barrier (probe)
    L.filter_ws = take(tdp_filter_workspace(nb));
    L.brow = take((size_t)nb * 4);
    L.bkey = take((size_t)nb * 4);
    L.ukey = take((size_t)nb * 4);
    L.skey = take((size_t)nb * 4);
    L.srow = take((size_t)nb * 4);
    L.radix = take(radix_ws_bytes(nb, 32, 4, 4));
    L.dkey = take((size_t)nb * 4);
    L.start = take((size_t)(nb + 1) * 4);
    L.table = take((size_t)L.nslots * 8);
    L.pord = take((size_t)std::max(1ll, n_probe) * 4);
    L.totals = take((size_t)L.Gmax * 8 * 2);
    L.total = off;
    return L;
}

} // namespace tdp

using namespace tdp;

extern "C" int64_t tdp_join_default_slots(int64_t n_keys)
{
    long long s = 8;
    while (s < 2 * n_keys)
        s <<= 1;
    return s;
}

extern "C" tdp_status tdp_join_build(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                                     int64_t n, const int64_t *d_n, int32_t key_col, int32_t payload_col, uint32_t flags,
                                     uint64_t *table, int64_t nslots, int32_t *d_status, tdp_stream_t stream)
{
    (void)flags;
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !table_ok(table, nslots) || key_col < 0 ||
        key_col >= ncols || payload_col >= ncols)
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
    const TableView tv = table_view(table, nslots);
    fill_empty_kernel<<<(unsigned)std::min<long long>((nslots / 2 + 255) / 256, (long long)num_sms() * 8), 256, 0,
                        s>>>((uint32_t *)table, nslots);
    if (n > 0) {
        // one thread per 4 rows (the kernel is not grid-strided)
        unsigned grid = (unsigned)((n + 1023) / 1024);
        join_build_kernel<<<grid, 256, 0, s>>>(ps, (const int32_t *)cols[key_col].data,
                                               payload_col >= 0 ? (const int32_t *)cols[payload_col].data : nullptr,
                                               n, (const long long *)d_n, (uint32_t *)table, tv.lgb, tv.steps,
                                               d_status);
    }
    return launch_status();
}

extern "C" size_t tdp_join_probe_workspace(int64_t n)
{
    // one look-back word per tile, sized for the smallest tile (1024 rows)
    long long tiles = (n + JP_THREADS * 4 - 1) / (JP_THREADS * 4);
    return align_up(16 + (size_t)tiles * 8, 256);
}

extern "C" tdp_status tdp_join_probe(const uint64_t *table, int64_t nslots, const tdp_col *cols, int32_t ncols,
                                     const tdp_pred *preds, int32_t npreds, int64_t n, const int32_t *sel,
                                     const int64_t *d_nsel, int32_t key_col, int32_t *out_probe_row,
                                     int32_t *out_payload, const int32_t *gather_cols, int32_t ngather,
                                     void *const *gather_out, int64_t capacity, int64_t *d_count, void *ws,
                                     size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !table_ok(table, nslots) || key_col < 0 ||
        key_col >= ncols || !d_count || capacity < 0 || (sel && !d_nsel))
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
    const TableView tv = table_view(table, nslots);
    const int32_t *key = (const int32_t *)cols[key_col].data;
    const long long *dn = (const long long *)d_nsel;
    long long *dc = (long long *)d_count;
    switch (probe_steps(ps)) {
    case 8: return launch_probe<8>(tv, ps, key, n, sel, dn, out_probe_row, out_payload, gs, capacity, dc, ws,
                                   d_status, s);
    case 4: return launch_probe<4>(tv, ps, key, n, sel, dn, out_probe_row, out_payload, gs, capacity, dc, ws,
                                   d_status, s);
    case 2: return launch_probe<2>(tv, ps, key, n, sel, dn, out_probe_row, out_payload, gs, capacity, dc, ws,
                                   d_status, s);
    default: return launch_probe<1>(tv, ps, key, n, sel, dn, out_probe_row, out_payload, gs, capacity, dc, ws,
                                    d_status, s);
    }
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
    if (n < 0 || n >= (1ll << 31) || !cols || !table || !table_ok(table, nslots) || key_col < 0 || key_col >= ncols ||
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
        GJStage sg;
        if (!make_gjstage(ps, as, cols[key_col].data, &sg))
            return TDP_ERR_INVALID_ARG;
        if ((st = launch_probe_agg(table_view(table, nslots), ps, sg, as, n, (const long long *)d_n, payload_lo, D,
                                   acc, d_status, s)) != TDP_OK)
            return st;
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

extern "C" size_t tdp_join_nm_workspace(int64_t n_build, int64_t n_probe)
{
    if (n_build < 0 || n_probe < 0)
        return 0;
    return nm_layout(n_build, n_probe).total;
}

extern "C" tdp_status tdp_join_nm(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                                  int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild, int32_t build_key_col,
                                  const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                                  int32_t nprobe_preds, int64_t n_probe, const int64_t *d_nprobe,
                                  int32_t probe_key_col, int32_t *out_probe_row, int32_t *out_build_row,
                                  int64_t capacity, int64_t *d_count, void *ws, size_t ws_bytes, int32_t *d_status,
                                  tdp_stream_t stream)
{
    if (n_build < 0 || n_build >= (1ll << 31) || n_probe < 0 || n_probe >= (1ll << 31) || !build_cols ||
        !probe_cols || build_key_col < 0 || build_key_col >= nbuild_cols || probe_key_col < 0 ||
        probe_key_col >= nprobe_cols || capacity < 0 || !d_count || (capacity > 0 && (!out_probe_row || !out_build_row)))
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
    const NmLayout L = nm_layout(n_build, n_probe);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws % 16) != 0)
        return TDP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    long long *cnt = (long long *)(w + L.counters);
    const long long nbm = std::max(1ll, (long long)n_build);
    if (cudaMemsetAsync(w + L.counters, 0, 256, s) != cudaSuccess ||
        cudaMemsetAsync(w + L.totals, 0, (size_t)L.Gmax * 16, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    // 1. qualifying build rows and their keys, sorted by key (stable)
    int32_t *brow = (int32_t *)(w + L.brow), *bkey = (int32_t *)(w + L.bkey);
    {
        const int32_t gcol = build_key_col;
        void *gout = bkey;
        GatherSet gs;
        if ((st = make_gatherset(build_cols, nbuild_cols, &gcol, 1, &gout, n_build, &gs)) != TDP_OK)
            return st;
        if ((st = filter_rows(bps, n_build, (const long long *)d_nbuild, brow, n_build, &cnt[0], &gs,
                              w + L.filter_ws, d_status, s)) != TDP_OK)
            return st;
    }
    uint32_t *ukey = (uint32_t *)(w + L.ukey), *skey = (uint32_t *)(w + L.skey), *srow = (uint32_t *)(w + L.srow);
    nm_pack_kernel<<<(unsigned)std::min<long long>((nbm + 255) / 256, (long long)num_sms() * 8), 256, 0, s>>>(
        bkey, n_build, &cnt[0], ukey);
    if ((st = launch_status()) != TDP_OK)
        return st;
    if ((st = radix_sort_pairs<uint32_t, uint32_t>(ukey, (const uint32_t *)brow, nbm, &cnt[0], 32, skey, srow,
                                                   w + L.radix, radix_ws_bytes(nbm, 32, 4, 4), d_status, s)) != TDP_OK)
        return st;
    // 2. runs of equal keys
    int32_t *dkey = (int32_t *)(w + L.dkey), *start = (int32_t *)(w + L.start);
    const uint32_t limit = spin_limit();
    {
        int G = 0, R = 1;
        if (!coop_grid_for((const void *)nm_runs_kernel, nbm, (long long)COOP_THREADS * NM_IPT, &G, &R))
            return TDP_ERR_CUDA;
        unsigned long long *tot = (unsigned long long *)(w + L.totals);
        unsigned *bar = (unsigned *)&cnt[2];
        long long nbmax = nbm;
        const long long *dnb = &cnt[0];
        long long *druns = &cnt[1];
        void *args[] = {(void *)&skey, (void *)&nbmax, (void *)&dnb, (void *)&R, (void *)&dkey, (void *)&start,
                        (void *)&druns, (void *)&tot, (void *)&bar, (void *)&d_status, (void *)&limit};
        if (cudaLaunchCooperativeKernel((const void *)nm_runs_kernel, dim3(G), dim3(COOP_THREADS), args, 0, s) !=
            cudaSuccess)
            return TDP_ERR_CUDA;
    }
    // 3. the distinct keys into the table, payload = run number
    uint64_t *table = (uint64_t *)(w + L.table);
    {
        tdp_col dc;
        dc.data = dkey;
        dc.dtype = TDP_I32;
        dc.has_bounds = 0;
        dc.n = nbm;
        dc.lo = dc.hi = 0;
        if ((st = tdp_join_build(&dc, 1, nullptr, 0, nbm, (const int64_t *)&cnt[1], 0, -1, TDP_JOIN_UNIQUE_BUILD,
                                 table, L.nslots, d_status, stream)) != TDP_OK)
            return st;
    }
    // 4. probe: count, then write
    if (n_probe == 0) {
        if (cudaMemsetAsync(d_count, 0, 8, s) != cudaSuccess)
            return TDP_ERR_CUDA;
        return launch_status();
    }
    {
        int G = 0, R = 1;
        if (!coop_grid_for((const void *)nm_probe_kernel, n_probe, (long long)COOP_THREADS * NM_IPT, &G, &R))
            return TDP_ERR_CUDA;
        TableView tv = table_view(table, L.nslots);
        const int32_t *pk = (const int32_t *)probe_cols[probe_key_col].data;
        long long np = n_probe;
        const long long *dnp = (const long long *)d_nprobe;
        int32_t *pord = (int32_t *)(w + L.pord);
        long long cap = capacity;
        long long *dc = (long long *)d_count;
        unsigned long long *tot = (unsigned long long *)(w + L.totals) + L.Gmax;
        unsigned *bar = (unsigned *)&cnt[3];
        const int32_t *cstart = start;
        const uint32_t *csrow = srow;
        void *args[] = {(void *)&tv, (void *)&pps, (void *)&pk, (void *)&np, (void *)&dnp, (void *)&R,
                        (void *)&cstart, (void *)&csrow, (void *)&pord, (void *)&out_probe_row,
                        (void *)&out_build_row, (void *)&cap, (void *)&dc, (void *)&tot, (void *)&bar,
                        (void *)&d_status, (void *)&limit};
        if (cudaLaunchCooperativeKernel((const void *)nm_probe_kernel, dim3(G), dim3(COOP_THREADS), args, 0, s) !=
            cudaSuccess)
            return TDP_ERR_CUDA;
    }
    return launch_status();
}
