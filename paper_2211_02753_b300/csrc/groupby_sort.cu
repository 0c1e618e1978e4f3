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
//  4. Reduce-by-key over the sorted pairs in one pass: each thread folds 8
//     consecutive pairs, the block scans (head count, running aggregates)
//     with the segmented operator (a, b) -> (a.h + b.h, b.h ? b.s : a.s (+) b.s),
//     tiles chain their carries by decoupled look-back, and the thread that
//     holds the last pair of a group writes the group (key fields unpacked,
//     aggregates finalised).  Groups come out in ascending key order.
#include "filter_api.cuh"
#include "groupby.cuh"
#include "radix.cuh"

namespace tdp {

constexpr int SR_THREADS = 256;
constexpr int SR_ITEMS = 8;
constexpr int SR_TILE = SR_THREADS * SR_ITEMS;
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
        for (int k = 0; k < ks.n; k++) {
            long long v[U];
#pragma unroll
            for (int u = 0; u < U; u++)
                v[u] = row[u] >= 0 ? load_int(ks.col[k], ks.dt[k], row[u]) : 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                unsigned long long f;
                if (kp.bounded[k]) {
                    long long d = v[u] - ks.lo[k];
                    if (row[u] >= 0 && (d < 0 || d >= ks.size[k])) {
                        bad = true;
                        d = 0;
                    }
                    f = (unsigned long long)d;
                } else {
                    const int w = kp.bits[k];
                    f = (unsigned long long)v[u] & field_mask(w);
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
                rows[i] = CARRY ? (V)slot_value(as, 1, row[u]) : (V)(positions ? i : row[u]);
            }
        }
    }
    if (bad)
        set_status(d_status, TDP_ERR_OVERFLOW);
}

// Look-back record of a tile.  The aggregate and the inclusive prefix live in
// separate fields so that a reader never sees a half-overwritten value: the
// fields selected by `flag` (1: aggregate, 2: inclusive) are final once the
// flag is visible (written with release, read with acquire).
struct __align__(16) SegRec {
    unsigned flag;
    unsigned h_agg;
    unsigned h_inc;
    unsigned pad;
    long long s_agg[SR_MAXS];
    long long s_inc[SR_MAXS];
};

template <int SL>
struct SegValT {
    unsigned h;
    long long s[SL];
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

__device__ __forceinline__ void store_key(void *out, int dt, long long pos, long long v)
{
    switch (dt) {
    case TDP_I8: ((int8_t *)out)[pos] = (int8_t)v; break;
    case TDP_U8: ((uint8_t *)out)[pos] = (uint8_t)v; break;
    case TDP_I32: ((int32_t *)out)[pos] = (int32_t)v; break;
    default: ((long long *)out)[pos] = v; break;
    }
}

template <typename K, typename V, int SL, bool CARRY>
__global__ void __launch_bounds__(SR_THREADS, SL <= 5 ? 2 : 1) seg_reduce_kernel(const K *__restrict__ keys,
                                                                const V *__restrict__ rows, long long n_max,
                                                                const long long *d_n, KeySet ks, KeyPack kp,
                                                                AggSet as, DenseOut out, long long cap,
                                                                long long *d_ngroups, SegRec *recs, unsigned *ticket,
                                                                int32_t *d_status, uint32_t limit)
{
    using SV = SegValT<SL>;
    __shared__ long long s_tile;
    __shared__ SV s_warp[SR_THREADS / 32];
    __shared__ SV s_carry;
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
        int s = threadIdx.x, op = as.sop[s] == TDP_AGG_COUNT ? TDP_AGG_SUM : as.sop[s];
        s_ops[s] = op;
        s_init[s] = op == TDP_AGG_MIN ? 0x7fffffffffffffffll : op == TDP_AGG_MAX ? (long long)0x8000000000000000ull : 0;
    }
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    // persistent: tiles are taken in ticket order until the input runs out
    for (;;) {
    if (threadIdx.x == 0)
        s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    const long long tile_base = tile * SR_TILE;
    if (tile_base >= n)
        return;
    const int NS = as.nslots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long i0 = tile_base + (long long)threadIdx.x * SR_ITEMS;
    int ops[SL];
#pragma unroll
    for (int j = 0; j < SL; j++)
        ops[j] = s_ops[j];

    // thread fold: (heads, aggregates since the last head)
    SV mine;
    mine.h = 0;
#pragma unroll
    for (int j = 0; j < SL; j++)
        mine.s[j] = s_init[j];
    K prev = (i0 > 0 && i0 - 1 < n) ? keys[i0 - 1] : (K)0;
    unsigned headmask = 0;
    for (int it = 0; it < SR_ITEMS; it++) {
        long long i = i0 + it;
        if (i >= n)
            break;
        K key = keys[i];
        bool head = (i == 0) || key != prev;
        prev = key;
        if (head) {
            headmask |= 1u << it;
            mine.h++;
#pragma unroll
            for (int j = 0; j < SL; j++)
                mine.s[j] = s_init[j];
        }
        if (CARRY) { // count + the carried value of slot 1
            mine.s[0] += 1;
            mine.s[1] = comb(ops[1], mine.s[1], (long long)rows[i]);
        } else {
            const long long row = (long long)rows[i];
#pragma unroll
            for (int j = 0; j < SL; j++)
                if (j < NS)
                    mine.s[j] = comb(ops[j], mine.s[j], slot_value(as, j, row));
        }
    }
    // warp inclusive scan
    SV inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        SV up;
        up.h = __shfl_up_sync(0xffffffffu, inc.h, o);
#pragma unroll
        for (int j = 0; j < SL; j++)
            up.s[j] = __shfl_up_sync(0xffffffffu, inc.s[j], o);
        if (lane >= o) {
            SV r;
            seg_combine(ops, NS, up, inc, r);
            inc = r;
        }
    }
    if (lane == 31)
        s_warp[warp] = inc;
    // lane-exclusive within the warp
    SV lex;
    lex.h = __shfl_up_sync(0xffffffffu, inc.h, 1);
#pragma unroll
    for (int j = 0; j < SL; j++)
        lex.s[j] = __shfl_up_sync(0xffffffffu, inc.s[j], 1);
    if (lane == 0) {
        lex.h = 0;
#pragma unroll
        for (int j = 0; j < SL; j++)
            lex.s[j] = s_init[j];
    }
    __syncthreads();
    if (warp == 0) {
        // tile aggregate = fold of the warp totals (every lane computes it)
        SV agg = s_warp[0];
        for (int w = 1; w < SR_THREADS / 32; w++) {
            SV r;
            seg_combine(ops, NS, agg, s_warp[w], r);
            agg = r;
        }
        SegRec *me = recs + tile;
        SV excl;
        excl.h = 0;
#pragma unroll
        for (int j = 0; j < SL; j++)
            excl.s[j] = s_init[j];
        if (tile == 0) {
            if (lane == 0) {
                me->h_inc = agg.h;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    if (j < NS)
                        me->s_inc[j] = agg.s[j];
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&me->flag), "r"(2u) : "memory");
            }
        } else {
            if (lane == 0) {
                me->h_agg = agg.h;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    if (j < NS)
                        me->s_agg[j] = agg.s[j];
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&me->flag), "r"(1u) : "memory");
            }
            // warp-parallel look-back: lane l reads the record of tile base-l;
            // the records up to the nearest inclusive one are folded in order
            // (earlier tiles first) and prepended to what was gathered so far.
            long long base = tile - 1;
            while (true) {
                const long long t = base - lane;
                unsigned f = 2;
                SV pv;
                pv.h = 0;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    pv.s[j] = s_init[j];
                if (t >= 0) {
                    const SegRec *pr = recs + t;
                    uint32_t polls = 0;
                    while (true) {
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(&pr->flag) : "memory");
                        if (f != 0)
                            break;
                        if (polls++ >= limit || ((polls & 63) == 0 && timed_out_already(d_status))) {
                            set_status(d_status, TDP_ERR_TIMEOUT);
                            break; // f == 0: treated as an (empty) inclusive record
                        }
                        __nanosleep(polls < 64 ? 20 : 200);
                    }
                    if (f != 0) {
                        pv.h = f == 2 ? *(volatile const unsigned *)&pr->h_inc : *(volatile const unsigned *)&pr->h_agg;
#pragma unroll
                        for (int j = 0; j < SL; j++)
                            if (j < NS)
                                pv.s[j] = f == 2 ? *(volatile const long long *)&pr->s_inc[j]
                                                 : *(volatile const long long *)&pr->s_agg[j];
                    }
                }
                const unsigned incl_mask = __ballot_sync(0xffffffffu, f != 1);
                const int k = incl_mask ? __ffs(incl_mask) - 1 : 31;
                SV w;
                w.h = 0;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    w.s[j] = s_init[j];
                for (int src = k; src >= 0; src--) { // k is warp-uniform
                    SV pj, r;
                    pj.h = __shfl_sync(0xffffffffu, pv.h, src);
#pragma unroll
                    for (int j = 0; j < SL; j++)
                        pj.s[j] = __shfl_sync(0xffffffffu, pv.s[j], src);
                    seg_combine(ops, NS, w, pj, r);
                    w = r;
                }
                SV r;
                seg_combine(ops, NS, w, excl, r);
                excl = r;
                if (incl_mask)
                    break;
                base -= 32;
            }
            if (lane == 0) {
                SV incl;
                seg_combine(ops, NS, excl, agg, incl);
                me->h_inc = incl.h;
#pragma unroll
                for (int j = 0; j < SL; j++)
                    if (j < NS)
                        me->s_inc[j] = incl.s[j];
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&me->flag), "r"(2u) : "memory");
            }
        }
        if (lane == 0)
            s_carry = excl;
    }
    __syncthreads();
    // carry into this thread = tile excl (+) warps before (+) lanes before
    SV carry = s_carry;
    for (int w = 0; w < warp; w++) {
        SV r;
        seg_combine(ops, NS, carry, s_warp[w], r);
        carry = r;
    }
    {
        SV r;
        seg_combine(ops, NS, carry, lex, r);
        carry = r;
    }
    // emit groups that end inside this thread's items
    long long g = (long long)carry.h - 1;
    SV run = carry;
    for (int it = 0; it < SR_ITEMS; it++) {
        long long i = i0 + it;
        if (i >= n)
            break;
        if (headmask >> it & 1) {
            g++;
#pragma unroll
            for (int j = 0; j < SL; j++)
                run.s[j] = s_init[j];
        }
        if (CARRY) {
            run.s[0] += 1;
            run.s[1] = comb(ops[1], run.s[1], (long long)rows[i]);
        } else {
            const long long row = (long long)rows[i];
#pragma unroll
            for (int j = 0; j < SL; j++)
                if (j < NS)
                    run.s[j] = comb(ops[j], run.s[j], slot_value(as, j, row));
        }
        bool last = (i == n - 1);
        K key = keys[i];
        if (!last)
            last = keys[i + 1] != key;
        if (last) {
            if (g >= 0 && g < cap) {
                unsigned long long packed = (unsigned long long)key;
                for (int k = 0; k < ks.n; k++) {
                    unsigned long long f = (packed >> kp.shift[k]) & field_mask(kp.bits[k]);
                    long long v;
                    if (kp.bounded[k]) {
                        v = ks.lo[k] + (long long)f;
                    } else {
                        int w = kp.bits[k];
                        if (ks.dt[k] != TDP_U8)
                            f ^= 1ull << (w - 1);
                        v = w >= 64 ? (long long)f : (long long)(f << (64 - w)) >> (64 - w);
                        if (ks.dt[k] == TDP_U8)
                            v = (long long)f;
                    }
                    store_key(s_out.key_out[k], s_out.key_dt[k], g, v);
                }
                // aggregates by slot (compile-time slot index; AVG needs the count)
#pragma unroll
                for (int j = 0; j < SL; j++) {
                    if (j >= NS)
                        continue;
                    for (int a = 0; a < s_as.n; a++) {
                        if (s_as.slot[a] != j)
                            continue;
                        long long v = run.s[j];
                        if (s_as.op[a] == TDP_AGG_AVG) {
                            long long c = run.s[0], sg = v > 0 ? 1 : (v < 0 ? -1 : 0);
                            v = (2 * v + sg * c) / (2 * c);
                        }
                        s_out.agg_out[a][g] = v;
                    }
                }
            }
            if (i == n - 1) {
                *d_ngroups = g + 1;
                if (g + 1 > cap)
                    set_status(d_status, TDP_ERR_CAPACITY);
            }
        }
    }
    __syncthreads(); // s_warp / s_carry are reused by the next tile
    }
}

// Few groups, several value slots: instead of the reduce gathering every
// slot input by row id (the groups' rows interleave, so each column would be
// read once per group, at gather latency), the slot values are written into
// sorted order.  (1) perm_invert: the sort carried input positions j; inv[j]
// = the sorted position of j, and the sorted payload becomes the identity.
// (2) perm_slots: the inputs in their own order (sequential reads) write
// each slot's value at inv[j]; the writes form one ascending stream per
// group, which L2 gathers into whole lines.  The reduce then streams them.
constexpr int PERM_MAX_KEY_BITS = 16; // at most 64K groups, so 64K write streams

template <typename V>
__global__ void perm_invert_kernel(V *sr, long long n, const long long *d_n, uint32_t *inv)
{
    const long long m = d_n ? min(*d_n, n) : n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        inv[(long long)sr[i]] = (uint32_t)i;
        sr[i] = (V)i;
    }
}

__global__ void perm_slots_kernel(AggSet as, long long n, const int32_t *sel, const long long *d_n,
                                  const uint32_t *__restrict__ inv, long long *__restrict__ perm, size_t stride)
{
    const long long m = d_n ? min(*d_n, n) : n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
        const long long row = sel ? sel[j] : j;
        const long long p = inv[j];
        for (int sl = 1; sl < as.nslots; sl++)
            perm[(size_t)(sl - 1) * stride + p] = slot_value(as, sl, row);
    }
}

static bool use_perm(int key_bits, bool carry) { return !carry && key_bits <= PERM_MAX_KEY_BITS; }

static size_t seg_ws(long long n)
{
    long long tiles = (n + SR_TILE - 1) / SR_TILE;
    return 256 + align_up((size_t)tiles * sizeof(SegRec), 256);
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
    if (n > 0)
        pack_keys_kernel<K, V, CARRY><<<grid, 256, 0, s>>>(ks, kp, as, n, rowsel, rowcount, pk, pr, perm, d_status);
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
    cudaMemsetAsync(segws, 0, seg_ws(n), s);
    long long tiles = (n + SR_TILE - 1) / SR_TILE;
    const unsigned sgrid = (unsigned)std::min<long long>(tiles, (long long)num_sms() * 3);
    auto launch = [&](auto kern) {
        kern<<<sgrid, SR_THREADS, 0, s>>>(sk, sr, n, rowcount, ks, kp, ras, out, capacity, (long long *)d_ngroups,
                                          (SegRec *)(segws + 256), (unsigned *)segws, d_status, spin_limit());
    };
    // accumulator slots carried through the scan: the smallest of 2, 4, 5, 9 that fits
    // (the carried state sets the registers, and so the blocks resident per SM)
    if (CARRY)
        launch(seg_reduce_kernel<K, V, 2, true>);
    else if (as.nslots <= 2)
        launch(seg_reduce_kernel<K, V, 2, false>);
    else if (as.nslots <= 4)
        launch(seg_reduce_kernel<K, V, 4, false>);
    else if (as.nslots <= 5)
        launch(seg_reduce_kernel<K, V, 5, false>);
    else
        launch(seg_reduce_kernel<K, V, SR_MAXS, false>);
    return launch_status();
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
