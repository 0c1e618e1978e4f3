// K3: onesweep LSD radix sort of (key, uint32 value) pairs, 8-bit digits.
//
//  1. One histogram pass reads every key once and counts all digit positions
//     (per-block shared-memory histograms; each lane adds runs of equal
//     digits among its own consecutive keys, so skewed or presorted digits
//     do not serialise on one counter).
//  2. A 256-thread kernel turns each digit position's histogram into
//     exclusive global offsets.
//  3. One scatter pass per digit.  A tile of 4096 pairs is copied into
//     shared memory and ranked there (each warp ranks its 512 pairs stably:
//     the lanes that share a digit come from nine ballots, a lane's rank is
//     their popc below it), publishes its per-digit counts, and every one of
//     the 256 threads finds its digit's offset by decoupled look-back over
//     earlier tiles (tile ids from an atomic ticket; waits bounded).  The
//     ranks become the tile's permutation into digit order, through which
//     the pairs are written out, so that the global writes of a digit run
//     are contiguous.
#include "radix.cuh"

namespace tdp {

constexpr unsigned RS_AGG = 1u << 30;
constexpr unsigned RS_INC = 2u << 30;
constexpr unsigned RS_VAL = (1u << 30) - 1;

// The lanes of the warp whose 9-bit value (an 8-bit digit, or 256 for "no
// element") equals this lane's: the AND over the bits of the ballot of the
// lanes that agree with this lane on that bit.
__device__ __forceinline__ unsigned digit_peers(unsigned d)
{
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; b++) {
        const unsigned bit = (d >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// Each lane reads 32 contiguous bytes of keys a step (two 16-byte loads when
// the keys are 16-byte aligned), so that enough bytes are in flight, and
// counts runs of equal digits among its own keys before one shared-memory
// atomic per run: skewed or presorted digits cost few atomics, random ones
// one per key, with no cross-lane ranking.
template <typename K, bool VEC>
__global__ void __launch_bounds__(RS_THREADS) radix_hist_kernel(const K *__restrict__ keys, long long n_max,
                                                                const long long *d_n, int passes,
                                                                unsigned *__restrict__ hist)
{
    constexpr int KPL = 32 / sizeof(K); // keys per lane per step
    __shared__ unsigned sh[8 * 256];
    for (int i = threadIdx.x; i < passes * 256; i += RS_THREADS)
        sh[i] = 0;
    __syncthreads();
    const long long n = d_n ? min(*d_n, n_max) : n_max;
    const long long step = (long long)gridDim.x * RS_THREADS * KPL;
    for (long long i0 = ((long long)blockIdx.x * RS_THREADS + threadIdx.x) * KPL; i0 < n; i0 += step) {
        K k[KPL];
        const int cnt = (int)min((long long)KPL, n - i0);
        if (VEC && cnt == KPL) {
            const uint4 a = __ldg((const uint4 *)(keys + i0)), b = __ldg((const uint4 *)(keys + i0) + 1);
            const unsigned w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < KPL; u++)
                k[u] = sizeof(K) == 4 ? (K)w[u] : (K)(((unsigned long long)w[2 * u + 1] << 32) | w[2 * u]);
        } else {
#pragma unroll
            for (int u = 0; u < KPL; u++)
                k[u] = u < cnt ? keys[i0 + u] : (K)0;
        }
        for (int p = 0; p < passes; p++) {
            unsigned run = (unsigned)((k[0] >> (8 * p)) & 0xff), c = 1;
#pragma unroll
            for (int u = 1; u < KPL; u++) {
                if (u >= cnt)
                    break;
                const unsigned d = (unsigned)((k[u] >> (8 * p)) & 0xff);
                if (d != run) {
                    atomicAdd(&sh[p * 256 + run], c);
                    run = d;
                    c = 0;
                }
                c++;
            }
            atomicAdd(&sh[p * 256 + run], c);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += RS_THREADS)
        if (sh[i])
            atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of 256 values held one per thread (256 threads).
__device__ __forceinline__ unsigned block_excl_scan_256(unsigned v, unsigned *s_tmp /* [8] */, unsigned *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_tmp[warp] = incl;
    __syncthreads();
    unsigned wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        unsigned t = s_tmp[w];
        wpre += w < warp ? t : 0;
        tot += t;
    }
    __syncthreads();
    if (total)
        *total = tot;
    return wpre + incl - v;
}

__global__ void radix_hist_scan_kernel(unsigned *hist)
{
    __shared__ unsigned tmp[8];
    unsigned *h = hist + blockIdx.x * 256;
    unsigned v = h[threadIdx.x];
    unsigned e = block_excl_scan_256(v, tmp, nullptr);
    h[threadIdx.x] = e;
}

__device__ __forceinline__ unsigned rs_wait(const unsigned *w, uint32_t limit, int32_t *d_status, bool *timed_out)
{
    unsigned s = ld_relaxed_u32(w);
    uint32_t polls = 0;
    while ((s >> 30) == 0) {
        if (polls++ >= limit || ((polls & 63) == 0 && timed_out_already(d_status))) {
            set_status(d_status, TDP_ERR_TIMEOUT);
            *timed_out = true;
            return s;
        }
        __nanosleep(polls < 64 ? 20 : 200);
        s = ld_relaxed_u32(w);
    }
    return s;
}

// 16-byte asynchronous global -> shared copy (L2 only), and its wait.
__device__ __forceinline__ void rs_cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ void rs_cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One onesweep digit pass.  The tile's pairs are copied into shared memory
// in input order (16-byte cp.async for a full tile of 16-byte aligned
// arrays), ranked there, and the ranks become a permutation: s_src[j] = the
// input index of the tile's j-th pair in digit order.  The write-out reads
// the pairs back through it, so a thread keeps only its 16 (digit, rank)
// words in registers and three blocks fit on an SM.
template <typename K, typename V>
__global__ void __launch_bounds__(RS_THREADS, 3) radix_scatter_kernel(const K *__restrict__ kin,
                                                                      const V *__restrict__ vin,
                                                                      K *__restrict__ kout, V *__restrict__ vout,
                                                                      long long n_max, const long long *d_n,
                                                                      int shift, const unsigned *__restrict__ offsets,
                                                                      unsigned *status, unsigned *ticket,
                                                                      int32_t *d_status, uint32_t limit, int vec)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    K *s_keys = (K *)rs_smem;                           // [RS_TILE], input order
    V *s_vals = (V *)(s_keys + RS_TILE);                // [RS_TILE], input order
    uint16_t *s_src = (uint16_t *)(s_vals + RS_TILE);   // [RS_TILE], digit order -> input index
    unsigned *s_whist = (unsigned *)(s_src + RS_TILE);  // [RS_WARPS][257]
    __shared__ unsigned s_dstart[256];
    __shared__ unsigned s_glob[256];
    __shared__ unsigned s_tmp[8];
    __shared__ long long s_tile;

    const long long n = d_n ? min(*d_n, n_max) : n_max;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned *wh = s_whist + warp * 257;
    // persistent: tiles are taken in ticket order until the input runs out
    for (;;) {
        if (threadIdx.x == 0)
            s_tile = atomicAdd(ticket, 1u);
        for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_THREADS)
            s_whist[i] = 0;
        __syncthreads();
        const long long tile = s_tile;
        const long long tile_base = tile * RS_TILE;
        if (tile_base >= n)
            return;
        const int m = (int)min((long long)RS_TILE, n - tile_base);
        // 1. the tile into shared memory, input order
        if (vec && m == RS_TILE) {
            constexpr int KCH = RS_TILE * (int)sizeof(K) / 16, VCH = RS_TILE * (int)sizeof(V) / 16;
            const char *gk = (const char *)(kin + tile_base), *gv = (const char *)(vin + tile_base);
            for (int c = threadIdx.x; c < KCH; c += RS_THREADS)
                rs_cp_async16((char *)s_keys + 16 * c, gk + 16 * c);
            for (int c = threadIdx.x; c < VCH; c += RS_THREADS)
                rs_cp_async16((char *)s_vals + 16 * c, gv + 16 * c);
            rs_cp_async_wait_all();
        } else {
            for (int p = threadIdx.x; p < m; p += RS_THREADS) {
                s_keys[p] = kin[tile_base + p];
                s_vals[p] = vin[tile_base + p];
            }
        }
        __syncthreads();
        // 2. stable rank within the warp's 512 pairs (digit 256: no pair)
        uint32_t dr[RS_ITEMS]; // digit | rank << 16
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) {
            const int p = warp * (RS_ITEMS * 32) + i * 32 + lane;
            const unsigned d = p < m ? (unsigned)((s_keys[p] >> shift) & 0xff) : 256u;
            const unsigned peers = digit_peers(d);
            const unsigned base = wh[d];
            dr[i] = d | (base + __popc(peers & lt)) << 16;
            __syncwarp();
            if ((peers & lt) == 0)
                wh[d] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit d = threadIdx.x: exclusive prefix over warps and tile count
        const int d = threadIdx.x;
        unsigned cnt = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            const unsigned c = s_whist[w * 257 + d];
            s_whist[w * 257 + d] = cnt;
            cnt += c;
        }
        const unsigned dstart = block_excl_scan_256(cnt, s_tmp, nullptr);
        s_dstart[d] = dstart;
        // decoupled look-back for this digit
        unsigned excl = 0;
        unsigned *my = status + tile * 256 + d;
        if (tile == 0) {
            st_relaxed_u32(my, RS_INC | cnt);
        } else {
            st_relaxed_u32(my, RS_AGG | cnt);
            long long t = tile - 1;
            while (t >= 0) {
                bool to = false;
                const unsigned s = rs_wait(status + t * 256 + d, limit, d_status, &to);
                excl += s & RS_VAL;
                if ((s >> 30) == 2 || to)
                    break;
                t--;
            }
            st_relaxed_u32(my, RS_INC | ((excl + cnt) & RS_VAL));
        }
        s_glob[d] = offsets[d] + excl;
        __syncthreads();
        // 3. the tile's permutation into digit order
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) {
            const unsigned dd = dr[i] & 0xffffu;
            if (dd < 256) {
                const unsigned lp = s_dstart[dd] + s_whist[warp * 257 + dd] + (dr[i] >> 16);
                s_src[lp] = (uint16_t)(warp * (RS_ITEMS * 32) + i * 32 + lane);
            }
        }
        __syncthreads();
        // 4. coalesced write-out: a digit's run is contiguous in the output
        for (int j = threadIdx.x; j < m; j += RS_THREADS) {
            const int p = s_src[j];
            const K key = s_keys[p];
            const unsigned dd = (unsigned)((key >> shift) & 0xff);
            const long long g = (long long)s_glob[dd] + (j - (long long)s_dstart[dd]);
            kout[g] = key;
            vout[g] = s_vals[p];
        }
        __syncthreads(); // shared staging is reused by the next tile
    }
}

size_t radix_ws_bytes(long long n, int key_bits, int key_bytes, int val_bytes)
{
    int P = radix_passes(key_bits);
    long long tiles = (n + RS_TILE - 1) / RS_TILE;
    size_t b = align_up((size_t)P * 256 * 4, 256) + 256 + align_up((size_t)P * tiles * 256 * 4, 256);
    b += align_up((size_t)n * key_bytes, 256) + align_up((size_t)n * val_bytes, 256);
    return b;
}

template <typename K, typename V>
tdp_status radix_sort_pairs(const K *keys_in, const V *vals_in, long long n_max, const long long *d_n,
                            int key_bits, K *keys_out, V *vals_out, void *ws, size_t ws_bytes,
                            int32_t *d_status, cudaStream_t s)
{
    if (key_bits < 1 || key_bits > (int)(8 * sizeof(K)) || n_max < 0 || n_max >= (1ll << 30))
        return TDP_ERR_INVALID_ARG;
    if (n_max == 0)
        return TDP_OK;
    if (ws_bytes < radix_ws_bytes(n_max, key_bits, sizeof(K), sizeof(V)))
        return TDP_ERR_WORKSPACE_TOO_SMALL;
    const int P = radix_passes(key_bits);
    const long long tiles = (n_max + RS_TILE - 1) / RS_TILE;
    char *p = (char *)ws;
    unsigned *hist = (unsigned *)p;
    p += align_up((size_t)P * 256 * 4, 256);
    unsigned *tickets = (unsigned *)p;
    p += 256;
    unsigned *status = (unsigned *)p;
    p += align_up((size_t)P * tiles * 256 * 4, 256);
    K *tmp_k = (K *)p;
    p += align_up((size_t)n_max * sizeof(K), 256);
    V *tmp_v = (V *)p;
    cudaMemsetAsync(ws, 0, (size_t)((char *)tmp_k - (char *)ws), s);
    constexpr int KPL = 32 / sizeof(K);
    const int hist_blocks =
        (int)std::min<long long>((n_max + RS_THREADS * KPL - 1) / (RS_THREADS * KPL), (long long)num_sms() * 4);
    if ((uintptr_t)keys_in % 16 == 0)
        radix_hist_kernel<K, true><<<hist_blocks, RS_THREADS, 0, s>>>(keys_in, n_max, d_n, P, hist);
    else
        radix_hist_kernel<K, false><<<hist_blocks, RS_THREADS, 0, s>>>(keys_in, n_max, d_n, P, hist);
    radix_hist_scan_kernel<<<P, 256, 0, s>>>(hist);
    const size_t smem = (size_t)RS_TILE * (sizeof(K) + sizeof(V) + 2) + RS_WARPS * 257 * 4;
    if (cudaFuncSetAttribute(radix_scatter_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return TDP_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, radix_scatter_kernel<K, V>, RS_THREADS, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return TDP_ERR_CUDA;
    const K *src_k = keys_in;
    const V *src_v = vals_in;
    // persistent grid: as many blocks as are resident at once
    const unsigned sgrid = (unsigned)std::min<long long>(tiles, (long long)num_sms() * per_sm);
    for (int pass = 0; pass < P; pass++) {
        bool to_out = ((P - 1 - pass) % 2) == 0;
        K *dk = to_out ? keys_out : tmp_k;
        V *dv = to_out ? vals_out : tmp_v;
        const int vec = (((uintptr_t)src_k | (uintptr_t)src_v) % 16) == 0;
        radix_scatter_kernel<K, V><<<sgrid, RS_THREADS, smem, s>>>(
            src_k, src_v, dk, dv, n_max, d_n, 8 * pass, hist + pass * 256, status + (size_t)pass * tiles * 256,
            tickets + pass, d_status, spin_limit(), vec);
        src_k = dk;
        src_v = dv;
    }
    return launch_status();
}

#define TDP_RADIX_INST(K, V)                                                                                  \
    template tdp_status radix_sort_pairs<K, V>(const K *, const V *, long long, const long long *, int, K *, V *,   \
                                               void *, size_t, int32_t *, cudaStream_t);
TDP_RADIX_INST(uint32_t, uint32_t)
TDP_RADIX_INST(unsigned long long, uint32_t)
TDP_RADIX_INST(uint32_t, unsigned long long)
TDP_RADIX_INST(unsigned long long, unsigned long long)
#undef TDP_RADIX_INST

} // namespace tdp

using namespace tdp;

extern "C" size_t tdp_sort_pairs_workspace(int64_t n, int32_t key_bits)
{
    if (key_bits < 1 || key_bits > 64 || n < 0)
        return 0;
    return radix_ws_bytes(n, key_bits, 8, 4);
}

extern "C" tdp_status tdp_sort_pairs(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t key_bits,
                                     uint64_t *keys_out, uint32_t *vals_out, void *ws, size_t ws_bytes,
                                     int32_t *d_status, tdp_stream_t stream)
{
    if (n < 0 || (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out || !ws)))
        return TDP_ERR_INVALID_ARG;
    if (n > 0 && (keys_in == (const uint64_t *)keys_out || vals_in == (const uint32_t *)vals_out))
        return TDP_ERR_INVALID_ARG;
    return radix_sort_pairs<unsigned long long, uint32_t>((const unsigned long long *)keys_in, vals_in, n, nullptr,
                                                          key_bits,
                                                (unsigned long long *)keys_out, vals_out, ws, ws_bytes, d_status,
                                                (cudaStream_t)stream);
}
