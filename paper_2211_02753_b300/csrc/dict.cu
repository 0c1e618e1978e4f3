// Order-preserving dictionary encoding of a string column (Sec. 2, Data
// Encoding: strings are stored as codes of a dictionary whose order is the
// strings' order, so that comparisons, sorts and groupings run on the codes).
//
// A string column is the usual offsets + bytes layout: row i is
// bytes[offsets[i] .. offsets[i+1]).  The code of a string is the number of
// distinct strings of the column that are smaller (bytewise unsigned
// lexicographic order, a proper prefix before its extensions), so
// code(a) < code(b) exactly when a < b.
//
//  1. every row's bytes, zero-padded to W = ceil(max_len / 8) big-endian
//     64-bit words, and its length;
//  2. the distinct strings: every row claims, or finds, its content's slot
//     in an open-addressing hash table of row ids (contents compared on a
//     hash match), so each row gets a representative row and each distinct
//     string one listed representative;
//  3. a stable LSD sort of the representatives only: by length, then by
//     word W-1, ..., word 0 (onesweep radix sort, each pass carrying the
//     row permutation, the count read on the device).  Zero padding alone
//     would tie "ab" with "ab\0"; the length pass, being the least
//     significant, breaks that tie with the shorter string first;
//  4. one cooperative pass over the sorted representatives: their codes are
//     their positions and each is copied into the dictionary (offsets from
//     the lengths' prefix sum); every other row then takes its
//     representative's code.
// (Sorting every row instead -- 25 digit passes over 10M rows for strings
// of up to 24 bytes -- took 5.6 ms where the rows hold 100K distinct
// strings; deduplicating first, 1.3 ms.)
#include <algorithm>

#include "coop.cuh"
#include "radix.cuh"

namespace tdp {

constexpr int DICT_MAX_LEN = 32;
constexpr int DICT_MAX_WORDS = DICT_MAX_LEN / 8;

// Row words (big-endian, zero padded) and lengths; rows longer than max_len
// are flagged and take the empty string's place in the order.
__global__ void dict_words_kernel(const int32_t *__restrict__ offsets, const uint8_t *__restrict__ bytes, long long n,
                                  int W, int max_len, unsigned long long *words, uint32_t *len_key, int32_t *d_status)
{
    bool too_long = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int32_t o = offsets[i];
        int len = offsets[i + 1] - o;
        if (len < 0 || len > max_len) {
            too_long = true;
            len = 0;
        }
        for (int k = 0; k < W; k++) {
            unsigned long long w = 0;
            for (int b = 0; b < 8; b++) {
                const int p = 8 * k + b;
                w = (w << 8) | (p < len ? bytes[o + p] : 0u);
            }
            words[(size_t)k * n + i] = w;
        }
        len_key[i] = (uint32_t)len;
    }
    if (too_long)
        set_status(d_status, TDP_ERR_OVERFLOW);
}

// keys[j] = words of word k for row perm[j] (the next LSD pass's keys), j <
// min(*d_m, n).
__global__ void dict_gather_kernel(const unsigned long long *words_k, const uint32_t *perm, long long n,
                                   const long long *d_m, unsigned long long *keys)
{
    const long long m = d_m ? min(*d_m, n) : n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
        keys[j] = words_k[perm[j]];
}

// Distinct strings by hashing: every row claims, or finds, the slot of its
// (words, length) in an open-addressing table of row ids (T slots, a power
// of two >= 2n, so a free slot always exists).  The content of the row
// that claimed a slot is already in memory (the words pass ran before), so
// a row that finds a claimed slot compares contents at once: equal means
// the same string (rep[row] = the claimer), else it moves to the next slot.
// Each claimer -- one row per distinct string -- is appended to the list of
// distinct rows with its length (the first sort pass's key); the count is
// *d_count.  Which of equal rows claims depends on timing; the codes and
// the dictionary do not (they depend on the contents only).
constexpr uint32_t DICT_EMPTY = 0xffffffffu;

__global__ void dict_insert_kernel(const unsigned long long *__restrict__ words, const uint32_t *__restrict__ len_key,
                                   long long n, int W, uint32_t *__restrict__ table, int lg_t, uint32_t *rep, uint32_t *list,
                                   uint32_t *list_len, unsigned long long *d_count, int32_t *d_status)
{
    const unsigned long long mask = (1ull << lg_t) - 1;
    const int lane = threadIdx.x & 31;
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += (long long)gridDim.x * blockDim.x) {
        const long long row = i0 + threadIdx.x;
        bool claimed = false;
        uint32_t len = 0;
        if (row < n) {
            len = len_key[row];
            unsigned long long w[DICT_MAX_WORDS];
            unsigned long long x = (len + 1) * 0x9E3779B97F4A7C15ull;
#pragma unroll
            for (int k = 0; k < DICT_MAX_WORDS; k++) {
                w[k] = k < W ? __ldg(words + (size_t)k * n + row) : 0;
                x = (x ^ w[k]) * 0xBF58476D1CE4E5B9ull;
                x ^= x >> 31;
            }
            unsigned long long sl = x >> (64 - lg_t);
            uint32_t r = DICT_EMPTY;
            for (unsigned long long step = 0; step <= mask; step++) {
                // a cached read: a stale "empty" only costs a CAS, which
                // returns the slot's row; contents never change here
                uint32_t cur = table[sl];
                if (cur == DICT_EMPTY) {
                    cur = atomicCAS(&table[sl], DICT_EMPTY, (uint32_t)row);
                    if (cur == DICT_EMPTY) {
                        r = (uint32_t)row;
                        claimed = true;
                        break;
                    }
                }
                bool same = __ldg(len_key + cur) == len;
#pragma unroll
                for (int k = 0; k < DICT_MAX_WORDS; k++)
                    same = same && (k >= W || __ldg(words + (size_t)k * n + cur) == w[k]);
                if (same) {
                    r = cur;
                    break;
                }
                sl = (sl + 1) & mask;
            }
            if (r == DICT_EMPTY) { // not reached: the table has more slots than rows
                set_status(d_status, TDP_ERR_CAPACITY);
                r = (uint32_t)row;
            }
            rep[row] = r;
        }
        // append the claimers (one atomic per warp)
        const unsigned cm = __ballot_sync(0xffffffffu, claimed);
        unsigned long long base = 0;
        if (lane == 0 && cm)
            base = atomicAdd(d_count, (unsigned long long)__popc(cm));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (claimed) {
            const unsigned long long at = base + __popc(cm & ((1u << lane) - 1u));
            list[at] = (uint32_t)row;
            list_len[at] = len;
        }
    }
}

// codes[row] = the code of row's representative (set by dict_codes_kernel
// for the representatives themselves).
__global__ void dict_fill_codes_kernel(const uint32_t *__restrict__ rep, long long n, int32_t *codes)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t r = rep[i];
        if (r != (uint32_t)i)
            codes[i] = codes[r];
    }
}

constexpr int DICT_IPT = 4; // sorted rows per thread per span

// Codes and dictionary from the sorted permutation of the distinct rows
// (cooperative): perm[0 .. m) with m = min(*d_m, n); the word arrays are
// indexed by row (stride n).  Codes are written for the rows in perm.
__global__ void __launch_bounds__(COOP_THREADS) dict_codes_kernel(
    const uint32_t *perm, long long n, const unsigned long long *d_m, int W, int rounds, const unsigned long long *words, const uint32_t *len_key,
    const int32_t *offsets, const uint8_t *bytes, int32_t *codes, int32_t *dict_offsets, uint8_t *dict_bytes,
    long long dict_cap, long long bytes_cap, long long *d_ndict, long long *d_nbytes, unsigned long long *totals,
    unsigned *barrier, int32_t *d_status, uint32_t limit)
{
    __shared__ unsigned long long s_red[COOP_THREADS / 32];
    __shared__ unsigned long long s_w64[COOP_THREADS / 32];
    __shared__ unsigned s_warp[COOP_THREADS / 32];
    const long long span = (long long)COOP_THREADS * DICT_IPT;
    const long long m = d_m ? min((long long)*d_m, n) : n;
    // the m items in equal contiguous ranges, one per block (the launch was
    // sized for n; rounds is recomputed for the range)
    const long long chunk = (m + gridDim.x - 1) / gridDim.x;
    const long long b0 = min(m, (long long)blockIdx.x * chunk), b1 = min(m, b0 + chunk);
    rounds = (int)((chunk + span - 1) / span);
    auto differs = [&](long long j) {
        if (j == 0)
            return true;
        const uint32_t a = perm[j], b = perm[j - 1];
        if (len_key[a] != len_key[b])
            return true;
        for (int k = 0; k < W; k++)
            if (words[(size_t)k * n + a] != words[(size_t)k * n + b])
                return true;
        return false;
    };
    // 1. heads (new codes) and their bytes, per block
    unsigned long long c = 0, cb = 0;
    for (int r = 0; r < rounds; r++) {
        const long long j0 = b0 + r * span + (long long)threadIdx.x * DICT_IPT;
#pragma unroll
        for (int e = 0; e < DICT_IPT; e++)
            if (j0 + e < b1 && differs(j0 + e)) {
                c++;
                cb += len_key[perm[j0 + e]];
            }
    }
    const unsigned long long tc = block_sum(c, s_red), tb = block_sum(cb, s_red);
    unsigned long long run_c, run_b;
    coop_block_prefix2(tc, tb, s_red, totals, barrier, limit, d_status, &run_c, &run_b);
    // 2. codes for every row, dictionary entries for the heads
    for (int r = 0; r < rounds; r++) {
        const long long j0 = b0 + r * span + (long long)threadIdx.x * DICT_IPT;
        unsigned h = 0, hb = 0;
#pragma unroll
        for (int e = 0; e < DICT_IPT; e++)
            if (j0 + e < b1 && differs(j0 + e)) {
                h |= 1u << e;
                hb += len_key[perm[j0 + e]];
            }
        unsigned tot;
        long long code = (long long)run_c + block_excl_scan(__popc(h), s_warp, &tot) - 1;
        unsigned long long totb;
        long long boff = (long long)run_b + block_excl_scan64(hb, s_w64, &totb);
        // the code of the run continuing into this thread's first row
        // starts before it: the previous row's code (code before any head)
        for (int e = 0; e < DICT_IPT; e++) {
            const long long j = j0 + e;
            if (j >= b1)
                break;
            const uint32_t row = perm[j];
            if (h >> e & 1u) {
                code++;
                const int len = (int)len_key[row];
                if (code < dict_cap)
                    dict_offsets[code] = (int32_t)boff;
                for (int p = 0; p < len; p++)
                    if (boff + p < bytes_cap)
                        dict_bytes[boff + p] = bytes[offsets[row] + p];
                boff += len;
            }
            codes[row] = (int32_t)code;
        }
        run_c += tot;
        run_b += totb;
        __syncthreads(); // s_warp / s_w64 reused by the next span's scans
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *d_ndict = (long long)run_c;
        *d_nbytes = (long long)run_b;
        if ((long long)run_c <= dict_cap)
            dict_offsets[run_c] = (int32_t)run_b;
        if ((long long)run_c > dict_cap || (long long)run_b > bytes_cap)
            set_status(d_status, TDP_ERR_CAPACITY);
    }
}

struct DictLayout {
    size_t counters, words, len_key, perm_a, perm_b, keys_a, keys_b, radix, radix_bytes, totals, rep, table, total;
    int W;
    int lg_t; // log2 of the distinct-string table's slots (>= 2n)
};

static DictLayout dict_layout(long long n, int max_len)
{
    DictLayout L;
    L.W = std::max(1, (max_len + 7) / 8);
    const long long m = std::max(1ll, n);
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align_up(off + b, 256);
        return o;
    };
    L.counters = take(256);
    L.words = take((size_t)L.W * m * 8);
    L.len_key = take((size_t)m * 4);
    L.perm_a = take((size_t)m * 4);
    L.perm_b = take((size_t)m * 4);
    L.keys_a = take((size_t)m * 8);
    L.keys_b = take((size_t)m * 8);
    L.radix_bytes = std::max(radix_ws_bytes(m, 64, 8, 4), radix_ws_bytes(m, 32, 4, 4));
    L.radix = take(L.radix_bytes);
    L.totals = take((size_t)8 * num_sms() * 8 * 8);
    L.rep = take((size_t)m * 4);
    L.lg_t = 6;
    while ((1ll << L.lg_t) < 2 * m)
        L.lg_t++;
    L.table = take((size_t)4 << L.lg_t);
    L.total = off;
    return L;
}

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_dict_encode_workspace(int64_t n, int32_t max_len)
{
    if (n < 0 || n >= (1ll << 31) || max_len < 1 || max_len > DICT_MAX_LEN)
        return 0;
    return dict_layout(n, max_len).total;
}

extern "C" tdp_status tdp_dict_encode(const int32_t *offsets, const uint8_t *bytes, int64_t n, int32_t max_len,
                                      int32_t *codes, int32_t *dict_offsets, uint8_t *dict_bytes, int64_t dict_cap,
                                      int64_t bytes_cap, int64_t *d_ndict, int64_t *d_nbytes, void *ws,
                                      size_t ws_bytes, int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || n >= (1ll << 31) || max_len < 1 || max_len > DICT_MAX_LEN || !offsets || !d_ndict || !d_nbytes ||
        dict_cap < 0 || bytes_cap < 0 || !dict_offsets || (n > 0 && (!bytes || !codes)) ||
        (bytes_cap > 0 && !dict_bytes))
        return TDP_ERR_INVALID_ARG;
    const DictLayout L = dict_layout(n, max_len);
    if (!ws || ws_bytes < L.total)
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws % 16) != 0)
        return TDP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    if (n == 0) {
        if (cudaMemsetAsync(d_ndict, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_nbytes, 0, 8, s) != cudaSuccess ||
            cudaMemsetAsync(dict_offsets, 0, 4, s) != cudaSuccess)
            return TDP_ERR_CUDA;
        return launch_status();
    }
    const int W = L.W;
    unsigned long long *words = (unsigned long long *)(w + L.words);
    uint32_t *len_key = (uint32_t *)(w + L.len_key);
    uint32_t *pa = (uint32_t *)(w + L.perm_a), *pb = (uint32_t *)(w + L.perm_b);
    unsigned long long *ka = (unsigned long long *)(w + L.keys_a), *kb = (unsigned long long *)(w + L.keys_b);
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
    if (cudaMemsetAsync(w + L.totals, 0, (size_t)8 * num_sms() * 8 * 8, s) != cudaSuccess ||
        cudaMemsetAsync(w + L.counters, 0, 256, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    dict_words_kernel<<<grid, 256, 0, s>>>(offsets, bytes, n, W, max_len, words, len_key, d_status);
    // the distinct strings: one representative row each, listed in pb with
    // their lengths (as 32-bit keys in kb), count in counters + 64
    uint32_t *rep = (uint32_t *)(w + L.rep);
    unsigned long long *d_cnt = (unsigned long long *)(w + L.counters + 64);
    if (cudaMemsetAsync(w + L.table, 0xff, (size_t)4 << L.lg_t, s) != cudaSuccess)
        return TDP_ERR_CUDA;
    dict_insert_kernel<<<grid, 256, 0, s>>>(words, len_key, n, W, (uint32_t *)(w + L.table), L.lg_t, rep, pb,
                                           (uint32_t *)kb, d_cnt, d_status);
    tdp_status st;
    const long long *dm = (const long long *)d_cnt;
    // sort the distinct rows, least significant first: the length (6 bits),
    // then word W-1 .. word 0
    if ((st = radix_sort_pairs<uint32_t, uint32_t>((uint32_t *)kb, pb, n, dm, 6, (uint32_t *)ka, pa, w + L.radix,
                                                   L.radix_bytes, d_status, s)) != TDP_OK)
        return st;
    for (int k = W - 1; k >= 0; k--) {
        dict_gather_kernel<<<grid, 256, 0, s>>>(words + (size_t)k * n, pa, n, dm, ka);
        if ((st = radix_sort_pairs<unsigned long long, uint32_t>(ka, pa, n, dm, 64, kb, pb, w + L.radix,
                                                                 L.radix_bytes, d_status, s)) != TDP_OK)
            return st;
        std::swap(pa, pb);
    }
    // pa: the distinct rows in order
    int G = 0, R = 1;
    if (!coop_grid_for((const void *)dict_codes_kernel, n, (long long)COOP_THREADS * DICT_IPT, &G, &R))
        return TDP_ERR_CUDA;
    long long nn = n, dc = dict_cap, bc = bytes_cap;
    const uint32_t *perm = pa;
    const unsigned long long *cnt = d_cnt;
    const unsigned long long *cw = words;
    const uint32_t *cl = len_key;
    unsigned long long *tot = (unsigned long long *)(w + L.totals);
    unsigned *bar = (unsigned *)(w + L.counters);
    long long *ndict = (long long *)d_ndict, *nbytes = (long long *)d_nbytes;
    const uint32_t limit = spin_limit();
    int Wv = W;
    void *args[] = {(void *)&perm, (void *)&nn, (void *)&cnt, (void *)&Wv, (void *)&R, (void *)&cw, (void *)&cl,
                    (void *)&offsets, (void *)&bytes, (void *)&codes, (void *)&dict_offsets, (void *)&dict_bytes,
                    (void *)&dc, (void *)&bc, (void *)&ndict, (void *)&nbytes, (void *)&tot, (void *)&bar,
                    (void *)&d_status, (void *)&limit};
    if (cudaLaunchCooperativeKernel((const void *)dict_codes_kernel, dim3(G), dim3(COOP_THREADS), args, 0, s) !=
        cudaSuccess)
        return TDP_ERR_CUDA;
    dict_fill_codes_kernel<<<grid, 256, 0, s>>>(rep, n, codes);
    return launch_status();
}
