// K4: sort-based group-by (tdp_groupby_agg, strategy SORT).
//
//  1. (optional) the WHERE predicates compact the input to a row-id list
//     (the filter kernel of filter.cu).
//  2. Pack each row's key tuple into one unsigned radix key: key 0 is the
//     most significant field; a bounded key takes ceil(log2(hi-lo+1)) bits
//     as key-lo, an unbounded one its full width with the sign bit flipped,
//     so unsigned order is lexicographic signed key order.  32-bit radix keys
//     when the fields fit, else 64-bit.
//  3. Onesweep radix sort of (packed key, payload) over the used bits only.
//     The payload is the row id, or -- when the query has a single value
//     aggregate besides COUNT -- that row's value itself (e.g. price*(100-disc)),
//     which spares the reduce a random gather per row.
//  4. Reduce-by-key over the sorted pairs (one cooperative launch): every
//     warp folds its run of pairs with the segmented operator
//     (a, b) -> (a.h + b.h, b.h ? b.s : a.s (+) b.s) over (head count,
//     running aggregates); after one grid barrier each warp takes the fold
//     of the runs before it as its carry and re-scans only the part of its
//     run in which groups end, and the lane that holds the last pair of a
//     group writes the group (key fields unpacked, aggregates finalised).
//     Groups come out in ascending key order.
#include "filter_api.cuh"
#include "groupby.cuh"
#include "radix.cuh"

namespace tdp {

constexpr int SR_THREADS = 256;
constexpr int SR_ITEMS = 8;
constexpr int SR_TILE = SR_THREADS * SR_ITEMS;
constexpr int SR_WTILE = 32 * SR_ITEMS; // rows a warp scans at a time
constexpr int SR_MAXS = TDP_MAX_AGGS + 1;

struct KeyPack {
    int32_t shift[TDP_MAX_KEYS];
    int32_t bits[TDP_MAX_KEYS];
    int32_t bounded[TDP_MAX_KEYS];
};

int key_field_bits(int dt, bool bounded, long long size)
{
    if (bounded) {
        int b = 1;
        while (b < 63 && (1ll << b) < size)
            b++;
        return b;
    }
    return 8 * dtype_size(dt);
}

int sort_key_bits(const KeySet &ks)
{
    int total = 0;
    for (int k = 0; k < ks.n; k++)
        total += key_field_bits(ks.dt[k], ks.size[k] > 0, ks.size[k]);
    return total <= 64 ? total : -1;
}

int sort_key_bits_desc(const tdp_col *keys, int32_t nkeys)
{
    int total = 0;
    for (int k = 0; k < nkeys; k++) {
        bool b = keys[k].has_bounds && keys[k].hi >= keys[k].lo;
        total += key_field_bits(keys[k].dtype, b, b ? keys[k].hi - keys[k].lo + 1 : 0);
    }
    return total <= 64 ? total : -1;
}

static KeyPack make_keypack(const KeySet &ks)
{
    KeyPack kp;
    int shift = 0;
    for (int k = TDP_MAX_KEYS - 1; k >= 0; k--) {
        if (k >= ks.n) {
            kp.shift[k] = kp.bits[k] = kp.bounded[k] = 0;
            continue;
        }
        kp.bounded[k] = ks.size[k] > 0;
        kp.bits[k] = key_field_bits(ks.dt[k], kp.bounded[k], ks.size[k]);
        kp.shift[k] = shift;
        shift += kp.bits[k];
    }
    return kp;
}

__device__ __forceinline__ unsigned long long field_mask(int bits)
{
    return bits >= 64 ? ~0ull : ((1ull << bits) - 1);
}

// Writes the packed key of every input row and its payload: the row id (or,
// with `positions`, the input position), or (CARRY) the value of
// accumulator slot 1 when that is the only value slot, so that the reduce
// streams it instead of gathering it by row id.
template <typename K, typename V, bool CARRY>
__global__ void pack_keys_kernel(KeySet ks, KeyPack kp, AggSet as, long long n, const int32_t *sel,
                                 const long long *d_nsel, K *keys, V *rows, bool positions, int32_t *d_status)
{
    const long long m = d_nsel ? min(*d_nsel, n) : n;
    bool bad = false;
    constexpr int U = 4; // rows in flight per thread: their loads are issued together
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += stride * U) {
        long long row[U];
        unsigned long long packed[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = i0 + u * stride;
            row[u] = i < m ? (sel ? sel[i] : i) : -1;
            packed[u] = 0;
        }
        // every key column (and the carried value) of the U rows is loaded
        // before any of them is used: one round trip after the row ids
        long long v[TDP_MAX_KEYS][U];
#pragma unroll
        for (int k = 0; k < TDP_MAX_KEYS; k++)
            if (k < ks.n) {
#pragma unroll
                for (int u = 0; u < U; u++)
                    v[k][u] = row[u] >= 0 ? load_int(ks.col[k], ks.dt[k], row[u]) : 0;
            }
        V cv[U];
        if (CARRY) {
#pragma unroll
            for (int u = 0; u < U; u++)
                cv[u] = row[u] >= 0 ? (V)slot_value(as, 1, row[u]) : (V)0;
        }
#pragma unroll
        for (int k = 0; k < TDP_MAX_KEYS; k++) {
            if (k >= ks.n)
                break;
#pragma unroll
            for (int u = 0; u < U; u++) {
                unsigned long long f;
                if (kp.bounded[k]) {
                    long long d = v[k][u] - ks.lo[k];
                    if (row[u] >= 0 && (d < 0 || d >= ks.size[k])) {
                        bad = true;
                        d = 0;
                    }
                    f = (unsigned long long)d;
                } else {
                    const int w = kp.bits[k];
                    f = (unsigned long long)v[k][u] & field_mask(w);
                    if (ks.dt[k] != TDP_U8)
                        f ^= 1ull << (w - 1);
                }
                packed[u] |= f << kp.shift[k];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = i0 + u * stride;
            if (i < m) {
                keys[i] = (K)packed[u];
                rows[i] = CARRY ? cv[u] : (V)(positions ? i : row[u]);
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
}

// Segmented fold of sorted rows: heads seen, and each slot's aggregate since
// the last head (the whole span's aggregate when no head was seen).
template <int SL>
struct SegValT {
    unsigned h;
    long long s[SL];
};

// A warp run's record: heads, each slot's aggregate since the last head,
// and before the first head (both over all rows when there is none).
template <int SL>
struct SegPreT {
    unsigned h;
    long long s[SL];
    long long p[SL];
};

__device__ __forceinline__ long long comb(int op, long long a, long long b)
{
    return op == TDP_AGG_MIN ? min(a, b) : op == TDP_AGG_MAX ? max(a, b) : a + b;
}

// a then b
template <int SL>
__device__ __forceinline__ void seg_combine(const int *ops, int NS, const SegValT<SL> &a, const SegValT<SL> &b,
                                            SegValT<SL> &r)
{
    r.h = a.h + b.h;
#pragma unroll
    for (int j = 0; j < SL; j++)
        if (j < NS)
            r.s[j] = b.h ? b.s[j] : comb(ops[j], a.s[j], b.s[j]);
}

template <int SL>
__device__ __forceinline__ void seg_identity(SegValT<SL> &v, const long long *init)
{
    v.h = 0;
#pragma unroll
    for (int j = 0; j < SL; j++)
        v.s[j] = init[j];
}

template <int SL>
__device__ __forceinline__ void seg_shfl_down(SegValT<SL> &v, int o)
{
    v.h = __shfl_down_sync(0xffffffffu, v.h, o);
#pragma unroll
    for (int j = 0; j < SL; j++)
        v.s[j] = __shfl_down_sync(0xffffffffu, v.s[j], o);
}

template <int SL>
__device__ __forceinline__ void seg_shfl_up(SegValT<SL> &v, int o)
{
    v.h = __shfl_up_sync(0xffffffffu, v.h, o);
#pragma unroll
    for (int j = 0; j < SL; j++)
        v.s[j] = __shfl_up_sync(0xffffffffu, v.s[j], o);
}

// Ordered fold of the 32 lanes' values (lane 0 first); the result is lane 0's.
template <typename SV>
__device__ __forceinline__ void seg_warp_fold(const int *ops, int NS, SV &v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        SV up = v, r;
        seg_shfl_down(up, o);
        seg_combine(ops, NS, v, up, r);
        if (lane + o < 32)
            v = r;
    }
}

__device__ __forceinline__ void store_key(void *out, int dt, long long pos, long long v)
{
    switch (dt) {
    case TDP_I8: ((int8_t *)out)[pos] = (int8_t)v; break;
    case TDP_U8: ((uint8_t *)out)[pos] = (uint8_t)v; break;
    case TDP_I32: ((int32_t *)out)[pos] = (int32_t)v; break;
    default: ((long long *)out)[pos] = v; break;
    }
}

// Where the reduce finds the slot values of sorted position i.
//   SEG_ROWS:  gathered by the row id the sort carried (slot_value).
//   SEG_CARRY: slot 1 is the carried value itself (slot 0 counts).
//   SEG_PERM:  slot j >= 1 at perm[(j - 1) * pstride + i], written into sorted
//              order beforehand (int64, SUM / MIN / MAX only).
enum SegMode { SEG_ROWS = 0, SEG_CARRY = 1, SEG_PERM = 2 };

struct SegSrc {
    const long long *perm;
    long long pstride;
};

template <typename K>
__device__ __forceinline__ void load4_keys(const K *p, K *k)
{
    if (sizeof(K) == 4) {
        const uint4 v = __ldg((const uint4 *)p);
        k[0] = (K)v.x, k[1] = (K)v.y, k[2] = (K)v.z, k[3] = (K)v.w;
    } else {
        const ulonglong2 a = __ldg((const ulonglong2 *)p), b = __ldg((const ulonglong2 *)p + 1);
        k[0] = (K)a.x, k[1] = (K)a.y, k[2] = (K)b.x, k[3] = (K)b.y;
    }
}

// Folds the sorted rows i0 .. i0 + SR_ITEMS - 1 that lie in [lo, end) into m
// and marks their heads in *headmask.  keys[i0 - 1] decides whether i0 is a
// head.  i0 is a multiple of SR_ITEMS.
template <typename K, typename V, int SL, int MODE>
__device__ __forceinline__ void seg_lane_fold(const K *__restrict__ keys, const V *__restrict__ rows,
                                              const AggSet &as, const SegSrc &src, long long i0, long long lo,
                                              long long end, const int *ops, const long long *init, int NS,
                                              SegValT<SL> &m, unsigned *headmask)
{
    K prev = (i0 > 0 && i0 < end) ? keys[i0 - 1] : (K)0;
    unsigned hm = 0;
#pragma unroll
    for (int half = 0; half < SR_ITEMS / 4; half++) {
        const long long b = i0 + half * 4;
        const bool full = b + 4 <= end;
        K kk[4];
        if (full) {
            load4_keys(keys + b, kk);
        } else {
#pragma unroll
            for (int it = 0; it < 4; it++)
                kk[it] = b + it < end ? keys[b + it] : (K)0;
        }
        // heads and active rows of these four
        unsigned hb = 0, act = 0;
#pragma unroll
        for (int it = 0; it < 4; it++) {
            const long long i = b + it;
            if (i < end) {
                const bool head = i == 0 || kk[it] != prev;
                prev = kk[it];
                if (i >= lo) {
                    act |= 1u << it;
                    if (head)
                        hb |= 1u << it;
                }
            }
        }
        hm |= hb << (half * 4);
        m.h += __popc(hb);
        if (MODE == SEG_PERM) {
            // slot by slot: four values live at a time
#pragma unroll
            for (int j = 0; j < SL; j++) {
                if (j >= NS)
                    continue;
                long long v[4];
                if (j == 0) {
                    v[0] = v[1] = v[2] = v[3] = 1;
                } else if (full) {
                    const longlong2 *q = (const longlong2 *)(src.perm + (j - 1) * src.pstride + b);
                    const longlong2 x = __ldg(q), y = __ldg(q + 1);
                    v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
                } else {
#pragma unroll
                    for (int it = 0; it < 4; it++)
                        v[it] = b + it < end ? src.perm[(j - 1) * src.pstride + b + it] : 0;
                }
                long long sj = m.s[j];
#pragma unroll
                for (int it = 0; it < 4; it++) {
                    if (!(act >> it & 1))
                        continue;
                    if (hb >> it & 1)
                        sj = init[j];
                    sj = comb(ops[j], sj, v[it]);
                }
                m.s[j] = sj;
            }
        } else {
#pragma unroll
            for (int it = 0; it < 4; it++) {
                if (!(act >> it & 1))
                    continue;
                const long long i = b + it;
                if (hb >> it & 1) {
#pragma unroll
                    for (int j = 0; j < SL; j++)
                        m.s[j] = init[j];
                }
                if (MODE == SEG_CARRY) {
                    m.s[0] += 1;
                    m.s[1] = comb(ops[1], m.s[1], (long long)rows[i]);
                } else {
                    const long long row = (long long)rows[i];
#pragma unroll
                    for (int j = 0; j < SL; j++)
                        if (j < NS)
                            m.s[j] = comb(ops[j], m.s[j], slot_value(as, j, row));
                }
            }
        }
    }
    *headmask = hm;
}

// Plain fold of the slot values of sorted rows [a, b) into this lane's acc
// (SUM, MIN and MAX commute, so every lane folds its own rows and the warp
// combines the lanes afterwards).  Lanes take 8 consecutive rows of each
// 256-row tile of the run that starts at ws.
template <typename K, typename V, int SL, int MODE>
__device__ __forceinline__ void seg_range_fold(const V *__restrict__ rows, const AggSet &as, const SegSrc &src,
                                               long long ws, long long a, long long b, const int *ops, int NS,
                                               long long *acc)
{
    const int lane = threadIdx.x & 31;
    if (a >= b)
        return;
    for (long long t = ws + (a - ws) / SR_WTILE * SR_WTILE; t < b; t += SR_WTILE) {
        const long long i0 = t + lane * SR_ITEMS;
        const long long lo = max(i0, a), hi = min(i0 + SR_ITEMS, b);
        if (lo >= hi)
            continue;
        acc[0] += hi - lo; // COUNT
        const bool full = lo == i0 && hi == i0 + SR_ITEMS;
        if (MODE == SEG_PERM || MODE == SEG_CARRY) {
#pragma unroll
            for (int j = 1; j < SL; j++) {
                if (j >= NS || (MODE == SEG_CARRY && j > 1))
                    continue;
                const long long *col = MODE == SEG_PERM ? src.perm + (j - 1) * src.pstride : (const long long *)rows;
                if (full) {
#pragma unroll
                    for (int q = 0; q < SR_ITEMS / 2; q++) {
                        const longlong2 x = __ldg((const longlong2 *)(col + i0) + q);
                        acc[j] = comb(ops[j], acc[j], x.x);
                        acc[j] = comb(ops[j], acc[j], x.y);
                    }
                } else {
                    for (long long i = lo; i < hi; i++)
                        acc[j] = comb(ops[j], acc[j], col[i]);
                }
            }
        } else {
            for (long long i = lo; i < hi; i++) {
                const long long row = (long long)rows[i];
#pragma unroll
                for (int j = 1; j < SL; j++)
                    if (j < NS)
                        acc[j] = comb(ops[j], acc[j], slot_value(as, j, row));
            }
        }
    }
}

// Writes group g: its key fields unpacked from the sorted key, and every
// aggregate from its accumulator slot (AVG from its sum and the count).
template <typename K, int SL>
__device__ __forceinline__ void emit_group(long long g, K key, const long long *acc, int NS, const KeySet &ks,
                                           const KeyPack &kp, const AggSet &as, const DenseOut &out)
{
    const unsigned long long packed = (unsigned long long)key;
    for (int k = 0; k < ks.n; k++) {
        unsigned long long f = (packed >> kp.shift[k]) & field_mask(kp.bits[k]);
        long long v;
        if (kp.bounded[k]) {
            v = ks.lo[k] + (long long)f;
        } else {
            const int w = kp.bits[k];
            if (ks.dt[k] != TDP_U8)
                f ^= 1ull << (w - 1);
            v = w >= 64 ? (long long)f : (long long)(f << (64 - w)) >> (64 - w);
            if (ks.dt[k] == TDP_U8)
                v = (long long)f;
        }
        store_key(out.key_out[k], out.key_dt[k], g, v);
    }
#pragma unroll
    for (int j = 0; j < SL; j++) {
        if (j >= NS)
            continue;
        for (int a = 0; a < as.n; a++) {
            if (as.slot[a] != j)
                continue;
            long long v = acc[j];
            if (as.op[a] == TDP_AGG_AVG) {
                const long long c = acc[0], sg = v > 0 ? 1 : (v < 0 ? -1 : 0);
                v = (2 * v + sg * c) / (2 * c);
            }
            out.agg_out[a][g] = v;
        }
    }
}

// Reduce-by-key of the sorted rows: one cooperative launch, every warp owning
// a contiguous run of whole 256-row tiles (the runs of a block are adjacent).
//   1. Each warp reads its run's keys and counts its heads (first and last
//      noted), then folds the slot values of the rows before the first head
//      and of the rows from the last head on (all rows when there is no
//      head) -- plain folds, the operators commute.  A block's (heads,
//      aggregates since the last head) is the ordered fold of its warps' and
//      goes to global memory.
//   2. One bounded grid barrier.
//   3. Each warp's carry is the ordered fold of everything before its run.
//      Lane 0 writes the group that ends inside the run before its first
//      head (carry + prefix), and, in the run that holds the final row, the
//      group from the last head to the end.  Groups that both start and end
//      inside the run lie between its first and last head: that span is
//      read again and scanned, and the lane holding a group's last row
//      writes it.
// Keys are read twice and every slot value once, except the values between
// a run's first and last head, which are read in step 3 only: with few
// groups the rows are streamed once; with many, 4 bytes a row more.  No warp
// waits on another except at the barrier.
template <typename K, typename V, int SL, int MODE>
__global__ void __launch_bounds__(SR_THREADS, SL <= 5 ? 2 : 1)
    seg_reduce_kernel(const K *__restrict__ keys, const V *__restrict__ rows, SegSrc src, long long n_max,
                      const long long *d_n, KeySet ks, KeyPack kp, AggSet as, DenseOut out, long long cap,
                      long long *d_ngroups, SegValT<SL> *recs, unsigned *barrier, int32_t *d_status, uint32_t limit)
{
    using SV = SegValT<SL>;
    using SP = SegPreT<SL>;
    constexpr int WARPS = SR_THREADS / 32;
    __shared__ SP s_wrec[WARPS];
    __shared__ long long s_wfirst[WARPS], s_wlast[WARPS];
    __shared__ SV s_red[WARPS];
    __shared__ int s_ops[SR_MAXS];
    __shared__ long long s_init[SR_MAXS];
    // parameter structs indexed with run-time indices live in shared memory
    // (indexing the kernel parameters directly would copy them to local memory)
    __shared__ AggSet s_as;
    __shared__ DenseOut s_out;
    if (threadIdx.x == 0) {
        s_as = as;
        s_out = out;
    }
    if (threadIdx.x < SR_MAXS) {
        const int s = threadIdx.x, op = as.sop[s] == TDP_AGG_COUNT ? TDP_AGG_SUM : as.sop[s];
        s_ops[s] = op;
        s_init[s] = op == TDP_AGG_MIN ? 0x7fffffffffffffffll : op == TDP_AGG_MAX ? (long long)0x8000000000000000ull : 0;
    }
    __syncthreads();
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    const int NS = as.nslots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ops[SL];
    long long init[SL];
#pragma unroll
    for (int j = 0; j < SL; j++) {
        ops[j] = s_ops[j];
        init[j] = s_init[j];
    }
    const long long tiles = (n + SR_WTILE - 1) / SR_WTILE;
    const long long nw = (long long)gridDim.x * WARPS;
    const long long per = (tiles + nw - 1) / nw;
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long ws = min(n, gw * per * SR_WTILE), we = min(n, ws + per * SR_WTILE);

    // 1a. the heads of the run (keys only): count, first, last; four tiles'
    // keys in flight per lane
    unsigned h = 0;
    long long first = -1, last = -1;
    constexpr int KT = 4;
    for (long long t0 = ws; t0 < we; t0 += KT * SR_WTILE) {
        K kk[KT][SR_ITEMS], pv[KT];
#pragma unroll
        for (int u = 0; u < KT; u++) {
            const long long i0 = t0 + u * SR_WTILE + lane * SR_ITEMS;
            pv[u] = (i0 > 0 && i0 < we) ? keys[i0 - 1] : (K)0;
            if (i0 + SR_ITEMS <= we) {
                load4_keys(keys + i0, kk[u]);
                load4_keys(keys + i0 + 4, kk[u] + 4);
            } else {
#pragma unroll
                for (int it = 0; it < SR_ITEMS; it++)
                    kk[u][it] = i0 + it < we ? keys[i0 + it] : (K)0;
            }
        }
#pragma unroll
        for (int u = 0; u < KT; u++) {
            const long long i0 = t0 + u * SR_WTILE + lane * SR_ITEMS;
            K prev = pv[u];
#pragma unroll
            for (int it = 0; it < SR_ITEMS; it++) {
                const long long i = i0 + it;
                if (i < we && (i == 0 || kk[u][it] != prev)) {
                    h++;
                    first = first < 0 ? i : first;
                    last = i;
                }
                prev = kk[u][it];
            }
        }
    }
    h = __reduce_add_sync(0xffffffffu, h);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long f = __shfl_xor_sync(0xffffffffu, first, o);
        first = first < 0 ? f : (f < 0 ? first : min(first, f));
        last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    }
    // 1b. the aggregates before the first head (all rows when there is none)
    // and after the last head: plain folds (SUM, MIN, MAX commute)
    long long pre[SL], suf[SL];
#pragma unroll
    for (int j = 0; j < SL; j++)
        pre[j] = suf[j] = init[j];
    seg_range_fold<K, V, SL, MODE>(rows, s_as, src, ws, ws, h ? first : we, ops, NS, pre);
    if (h)
        seg_range_fold<K, V, SL, MODE>(rows, s_as, src, ws, last, we, ops, NS, suf);
#pragma unroll
    for (int j = 0; j < SL; j++) {
        if (j >= NS)
            continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pre[j] = comb(ops[j], pre[j], __shfl_xor_sync(0xffffffffu, pre[j], o));
            suf[j] = comb(ops[j], suf[j], __shfl_xor_sync(0xffffffffu, suf[j], o));
        }
    }
    if (lane == 0) {
        SP &w = s_wrec[warp];
        w.h = h;
#pragma unroll
        for (int j = 0; j < SL; j++) {
            w.p[j] = pre[j];
            w.s[j] = h ? suf[j] : pre[j];
        }
        s_wfirst[warp] = first;
        s_wlast[warp] = last;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        SV b;
        seg_identity(b, init);
        for (int w = 0; w < WARPS; w++) {
            SV x, r;
            x.h = s_wrec[w].h;
#pragma unroll
            for (int j = 0; j < SL; j++)
                x.s[j] = s_wrec[w].s[j];
            seg_combine(ops, NS, b, x, r);
            b = r;
        }
        recs[blockIdx.x] = b;
    }
    grid_barrier(barrier, gridDim.x, limit, d_status);

    // 3. carry: thread t folds the records of blocks [t * q, (t + 1) * q)
    // before this one, then the lanes and warps are folded in order, then
    // the warps of this block before this one
    SV carry;
    {
        const int nb = blockIdx.x, q = (nb + SR_THREADS - 1) / SR_THREADS;
        SV part;
        seg_identity(part, init);
        const int r0 = threadIdx.x * q, r1 = min(nb, r0 + q);
        for (int r = r0; r < r1; r++) {
            SV rec, x;
            rec.h = __ldcg(&recs[r].h);
#pragma unroll
            for (int j = 0; j < SL; j++)
                rec.s[j] = j < NS ? __ldcg(&recs[r].s[j]) : init[j];
            seg_combine(ops, NS, part, rec, x);
            part = x;
        }
        seg_warp_fold(ops, NS, part);
        if (lane == 0)
            s_red[warp] = part;
        __syncthreads();
        seg_identity(carry, init);
        for (int w = 0; w < WARPS; w++) {
            SV x;
            seg_combine(ops, NS, carry, s_red[w], x);
            carry = x;
        }
        for (int w = 0; w < warp; w++) {
            SV x, y;
            x.h = s_wrec[w].h;
#pragma unroll
            for (int j = 0; j < SL; j++)
                x.s[j] = s_wrec[w].s[j];
            seg_combine(ops, NS, carry, x, y);
            carry = y;
        }
    }
    if (ws >= n)
        return;
    const SP &me = s_wrec[warp];
    const long long f = s_wfirst[warp], l = s_wlast[warp];
    const bool holds_end = we == n;
    if (lane == 0) {
        if ((me.h > 0 || holds_end) && carry.h > 0) {
            // the group open at the run's start: carry + the rows before the first head
            long long v[SL];
#pragma unroll
            for (int j = 0; j < SL; j++)
                v[j] = j < NS ? comb(ops[j], carry.s[j], me.p[j]) : 0;
            const long long g = (long long)carry.h - 1;
            if (g < cap)
                emit_group<K, SL>(g, me.h > 0 ? keys[f - 1] : keys[n - 1], v, NS, ks, kp, s_as, s_out);
        }
        if (holds_end) {
            const long long total = (long long)carry.h + me.h;
            if (me.h > 0 && total - 1 < cap) // the group from the last head to the final row
                emit_group<K, SL>(total - 1, keys[n - 1], me.s, NS, ks, kp, s_as, s_out);
            *d_ngroups = total;
            if (total > cap)
                set_status(d_status, TDP_ERR_CAPACITY);
        }
    }
    if (me.h < 2)
        return;
    // groups that start and end inside the run: rows [f, l), scanned from the
    // tile that holds f; rows before f are skipped (their sum is in no such group)
    SV wcarry;
    seg_identity(wcarry, init);
    wcarry.h = carry.h;
    for (long long t = ws + (f - ws) / SR_WTILE * SR_WTILE; t < l; t += SR_WTILE) {
        const long long i0 = t + lane * SR_ITEMS;
        SV mine;
        seg_identity(mine, init);
        unsigned headmask;
        seg_lane_fold<K, V, SL, MODE>(keys, rows, s_as, src, i0, f, l, ops, init, NS, mine, &headmask);
        SV inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            SV up = inc, r;
            seg_shfl_up(up, o);
            seg_combine(ops, NS, up, inc, r);
            if (lane >= o)
                inc = r;
        }
        SV lex = inc, total = inc;
        seg_shfl_up(lex, 1);
        if (lane == 0)
            seg_identity(lex, init);
        total.h = __shfl_sync(0xffffffffu, inc.h, 31);
#pragma unroll
        for (int j = 0; j < SL; j++)
            total.s[j] = __shfl_sync(0xffffffffu, inc.s[j], 31);
        SV run;
        seg_combine(ops, NS, wcarry, lex, run);
        {
            SV x;
            seg_combine(ops, NS, wcarry, total, x);
            wcarry = x;
        }
        // write the groups that end inside this lane's rows (all end before l)
        long long g = (long long)run.h - 1;
        for (int it = 0; it < SR_ITEMS; it++) {
            const long long i = i0 + it;
            if (i >= l)
                break;
            if (i < f)
                continue;
            if (headmask >> it & 1) {
                g++;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    run.s[j] = init[j];
            }
            if (MODE == SEG_CARRY) {
                run.s[0] += 1;
                run.s[1] = comb(ops[1], run.s[1], (long long)rows[i]);
            } else if (MODE == SEG_PERM) {
                run.s[0] += 1;
#pragma unroll
                for (int j = 1; j < SL; j++)
                    if (j < NS)
                        run.s[j] = comb(ops[j], run.s[j], src.perm[(j - 1) * src.pstride + i]);
            } else {
                const long long row = (long long)rows[i];
#pragma unroll
                for (int j = 0; j < SL; j++)
                    if (j < NS)
                        run.s[j] = comb(ops[j], run.s[j], slot_value(s_as, j, row));
            }
            const K key = keys[i];
            if (keys[i + 1] != key && g < cap)
                emit_group<K, SL>(g, key, run.s, NS, ks, kp, s_as, s_out);
        }
    }
}

// Few groups, several value slots: instead of the reduce gathering every
// slot input by row id (the groups' rows interleave, so each column would be
// read once per group, at gather latency), the slot values are written into
// sorted order.  (1) perm_invert: the sort carried input positions j; inv[j]
// = the sorted position of j.  (2) perm_slots: the inputs in their own
// order (sequential reads) write each slot's value at inv[j]; the writes
// form one ascending stream per group, which L2 gathers into whole lines.
// The reduce then streams them (SEG_PERM) and reads no payload.
constexpr int PERM_MAX_KEY_BITS = 16; // at most 64K groups, so 64K write streams

template <typename V>
__global__ void perm_invert_kernel(const V *__restrict__ sr, long long n, const long long *d_n, uint32_t *inv)
{
    constexpr int U = 4; // positions in flight per thread
    const long long m = d_n ? min(*d_n, n) : n;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += step * U) {
        long long j[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            j[u] = i0 + u * step < m ? (long long)sr[i0 + u * step] : -1;
#pragma unroll
        for (int u = 0; u < U; u++)
            if (j[u] >= 0)
                inv[j[u]] = (uint32_t)(i0 + u * step);
    }
}

__global__ void perm_slots_kernel(AggSet as, long long n, const int32_t *sel, const long long *d_n,
                                  const uint32_t *__restrict__ inv, long long *__restrict__ perm, size_t stride)
{
    constexpr int U = 4; // rows in flight per thread
    const long long m = d_n ? min(*d_n, n) : n;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; j0 < m; j0 += step * U) {
        long long row[U], p[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long j = j0 + u * step;
            row[u] = j < m ? (sel ? sel[j] : j) : -1;
            p[u] = j < m ? (long long)inv[j] : 0;
        }
        for (int sl = 1; sl < as.nslots; sl++) {
            long long v[U];
#pragma unroll
            for (int u = 0; u < U; u++)
                v[u] = row[u] >= 0 ? slot_value(as, sl, row[u]) : 0;
#pragma unroll
            for (int u = 0; u < U; u++)
                if (row[u] >= 0)
                    perm[(size_t)(sl - 1) * stride + p[u]] = v[u];
        }
    }
}

static bool use_perm(int key_bits, bool carry) { return !carry && key_bits <= PERM_MAX_KEY_BITS; }

// Barrier word + one record per block of the reduce (at most one block per
// SR_TILE rows).
static size_t seg_ws(long long n)
{
    long long tiles = (n + SR_TILE - 1) / SR_TILE;
    return 256 + align_up((size_t)tiles * sizeof(SegValT<SR_MAXS>), 256);
}

size_t sort_groupby_ws(long long n, int nkeys, int naggs, int key_bits)
{
    (void)nkeys;
    int kb = key_bits <= 32 ? 4 : 8;
    const int vb = 8; // payload: uint32 row id, or the carried int64 value
    size_t b = align_up((size_t)n * 4, 256);                         // filtered row ids
    b += 256;                                                         // filtered count
    b += 2 * align_up((size_t)n * kb, 256) + 2 * align_up((size_t)n * vb, 256); // packed pairs, sorted pairs
    b += radix_ws_bytes(n, key_bits, kb, vb);
    b += seg_ws(n);
    b += tdp_filter_workspace(n);
    if (key_bits <= PERM_MAX_KEY_BITS) // inverse positions + one int64 array per value slot
        b += align_up((size_t)n * 4, 256) + (size_t)naggs * align_up((size_t)n * 8, 256);
    return b;
}

template <typename K, typename V, bool CARRY>
static tdp_status sort_groupby_impl(const PredSet &ps, const KeySet &ks, int key_bits, const AggSet &as, long long n,
                                    const int32_t *sel, const int64_t *d_nsel, const DenseOut &out,
                                    long long capacity, int64_t *d_ngroups, void *ws, size_t ws_bytes,
                                    int32_t *d_status, cudaStream_t s)
{
    char *p = (char *)ws;
    int32_t *fsel = (int32_t *)p;
    p += align_up((size_t)n * 4, 256);
    long long *fcount = (long long *)p;
    p += 256;
    K *pk = (K *)p;
    p += align_up((size_t)n * sizeof(K), 256);
    K *sk = (K *)p;
    p += align_up((size_t)n * sizeof(K), 256);
    V *pr = (V *)p;
    p += align_up((size_t)n * 8, 256);
    V *sr = (V *)p;
    p += align_up((size_t)n * 8, 256);
    void *rws = p;
    size_t rws_bytes = radix_ws_bytes(n, key_bits, sizeof(K), 8);
    p += rws_bytes;
    char *segws = p;
    p += seg_ws(n);
    void *fws = p;
    p += tdp_filter_workspace(n);
    const bool perm = use_perm(key_bits, CARRY);
    uint32_t *inv = (uint32_t *)p;
    long long *pslots = nullptr;
    const size_t pstride = align_up((size_t)n * 8, 256) / 8;
    if (perm) {
        p += align_up((size_t)n * 4, 256);
        pslots = (long long *)p;
    }

    const int32_t *rowsel = sel;
    const long long *rowcount = (const long long *)d_nsel;
    if (ps.n > 0) {
        if (sel)
            return TDP_ERR_INVALID_ARG; // predicates over a row list: filter first
        tdp_status st = filter_rows(ps, n, (const long long *)d_nsel, fsel, n, fcount, nullptr, fws, d_status, s);
        if (st != TDP_OK)
            return st;
        rowsel = fsel;
        rowcount = fcount;
    }
    KeyPack kp = make_keypack(ks);
    int grid = (int)std::max(1ll, std::min<long long>((n + 255) / 256, (long long)num_sms() * 8));
    if (n > 0) {
        // grid-stride pack: one wave of resident blocks, so that no block
        // starts after the others have finished their share
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_keys_kernel<K, V, CARRY>, 256, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const int pgrid = (int)std::max(1ll, std::min<long long>((n + 255) / 256, (long long)num_sms() * per_sm));
        pack_keys_kernel<K, V, CARRY><<<pgrid, 256, 0, s>>>(ks, kp, as, n, rowsel, rowcount, pk, pr, perm, d_status);
    }
    tdp_status st = radix_sort_pairs<K, V>(pk, pr, n, rowcount, key_bits, sk, sr, rws, rws_bytes, d_status, s);
    if (st != TDP_OK)
        return st;
    cudaMemsetAsync(d_ngroups, 0, 8, s);
    if (n == 0)
        return launch_status();
    AggSet ras = as; // the aggregates as the reduce reads them
    if (perm) {
        perm_invert_kernel<V><<<grid, 256, 0, s>>>(sr, n, rowcount, inv);
        perm_slots_kernel<<<grid, 256, 0, s>>>(as, n, rowsel, rowcount, inv, pslots, pstride);
        for (int sl = 1; sl < as.nslots; sl++) {
            ras.sa[sl] = pslots + (size_t)(sl - 1) * pstride;
            ras.sadt[sl] = TDP_I64;
            if (ras.sop[sl] == TDP_AGG_SUM_MUL_KMINUS)
                ras.sop[sl] = TDP_AGG_SUM; // the stored value is already a * (k - b)
        }
    }
    cudaMemsetAsync(segws, 0, 256, s);
    // cooperative: at most two blocks per SM (16 warps streaming), at most one
    // block per SR_TILE rows
    const long long want = (n + SR_TILE - 1) / SR_TILE;
    const uint32_t limit = spin_limit();
    const SegSrc ssrc{pslots, (long long)pstride};
    auto launch = [&](auto kern, auto *recs) -> tdp_status {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SR_THREADS, 0) != cudaSuccess || per_sm < 1)
            return TDP_ERR_CUDA;
        const int G = (int)std::min<long long>(want, (long long)std::min(per_sm, 2) * num_sms());
        unsigned *barrier = (unsigned *)segws;
        const K *kk = sk;
        const V *rr = sr;
        long long *ng = (long long *)d_ngroups;
        void *args[] = {(void *)&kk, (void *)&rr, (void *)&ssrc, (void *)&n, (void *)&rowcount, (void *)&ks, (void *)&kp,
                        (void *)&ras, (void *)&out, (void *)&capacity, (void *)&ng, (void *)&recs,
                        (void *)&barrier, (void *)&d_status, (void *)&limit};
        if (cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(SR_THREADS), args, 0, s) != cudaSuccess)
            return TDP_ERR_CUDA;
        return launch_status();
    };
    // accumulator slots carried through the scan: the smallest of 2, 4, 5, 9 that fits
    // (the carried state sets the registers, and so the blocks resident per SM)
    if (CARRY)
        return launch(seg_reduce_kernel<K, V, 2, SEG_CARRY>, (SegValT<2> *)(segws + 256));
    auto by_slots = [&](auto mode) -> tdp_status {
        constexpr int M = decltype(mode)::value;
        if (as.nslots <= 2)
            return launch(seg_reduce_kernel<K, V, 2, M>, (SegValT<2> *)(segws + 256));
        if (as.nslots <= 4)
            return launch(seg_reduce_kernel<K, V, 4, M>, (SegValT<4> *)(segws + 256));
        if (as.nslots <= 5)
            return launch(seg_reduce_kernel<K, V, 5, M>, (SegValT<5> *)(segws + 256));
        return launch(seg_reduce_kernel<K, V, SR_MAXS, M>, (SegValT<SR_MAXS> *)(segws + 256));
    };
    return perm ? by_slots(std::integral_constant<int, SEG_PERM>()) : by_slots(std::integral_constant<int, SEG_ROWS>());
}

tdp_status sort_groupby_run(const PredSet &ps, const KeySet &ks, int key_bits, const AggSet &as, long long n,
                            const int32_t *sel, const int64_t *d_nsel, const DenseOut &out, long long capacity,
                            int64_t *d_ngroups, void *ws, size_t ws_bytes, int32_t *d_status, cudaStream_t s)
{
    // One value slot besides COUNT: carry the value through the sort (8-byte
    // payload) so that the reduce streams it; otherwise carry row ids.
    const bool carry = as.nslots == 2;
    if (key_bits <= 32)
        return carry ? sort_groupby_impl<uint32_t, unsigned long long, true>(ps, ks, key_bits, as, n, sel, d_nsel,
                                                                             out, capacity, d_ngroups, ws, ws_bytes,
                                                                             d_status, s)
                     : sort_groupby_impl<uint32_t, uint32_t, false>(ps, ks, key_bits, as, n, sel, d_nsel, out,
                                                                    capacity, d_ngroups, ws, ws_bytes, d_status, s);
    return carry ? sort_groupby_impl<unsigned long long, unsigned long long, true>(ps, ks, key_bits, as, n, sel,
                                                                                   d_nsel, out, capacity, d_ngroups,
                                                                                   ws, ws_bytes, d_status, s)
                 : sort_groupby_impl<unsigned long long, uint32_t, false>(ps, ks, key_bits, as, n, sel, d_nsel, out,
                                                                          capacity, d_ngroups, ws, ws_bytes, d_status,
                                                                          s);
}

} // namespace tdp
