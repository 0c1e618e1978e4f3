// Shared device helpers of the tdp kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tdp.h"

#define TDP_MAX_PREDS 8
#define TDP_MAX_GATHER 8
#define TDP_MAX_KEYS 4
#define TDP_MAX_AGGS 8

namespace tdp {

// ---------------------------------------------------------------- host side

// Current bounded-wait limit (polls) passed to every kernel that spins.
uint32_t spin_limit();

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int dtype_size(int dt)
{
    switch (dt) {
    case TDP_I8:
    case TDP_U8: return 1;
    case TDP_BF16: return 2;
    case TDP_I32:
    case TDP_F32: return 4;
    case TDP_I64: return 8;
    default: return 0;
    }
}

inline bool is_int_dtype(int dt) { return dt == TDP_I8 || dt == TDP_U8 || dt == TDP_I32 || dt == TDP_I64; }

inline tdp_status launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TDP_OK : TDP_ERR_CUDA;
}

int num_sms();

// Predicates as kernel parameters (values, not pointers to host memory).
struct PredSet {
    const void *col[TDP_MAX_PREDS];
    int32_t dt[TDP_MAX_PREDS];
    int32_t cmp[TDP_MAX_PREDS];
    long long lit[TDP_MAX_PREDS];
    int32_t vec_ok[TDP_MAX_PREDS]; // column base 16-byte aligned
    // Each comparison as a closed range test over the column's own type:
    // holds(v) = (lo <= v <= hi) != neg, with lo/hi clamped to the type's
    // range (an empty range is the full range with neg set: never true).
    long long lo[TDP_MAX_PREDS], hi[TDP_MAX_PREDS];
    int32_t neg[TDP_MAX_PREDS];
    int32_t n;
};

void pred_range(int dt, int cmp, long long lit, long long *lo, long long *hi, int32_t *neg);

// Validates `preds` against `cols` and fills a PredSet.
tdp_status make_predset(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds, int64_t n,
                        PredSet *out);

// ---------------------------------------------------------------- device side

__device__ __forceinline__ int dtype_size_dev(int dt)
{
    return dt == TDP_I64 ? 8 : (dt == TDP_I32 || dt == TDP_F32) ? 4 : dt == TDP_BF16 ? 2 : 1;
}

__device__ __forceinline__ void set_status(int32_t *s, int32_t code)
{
    if (s)
        atomicOr(s, code);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ long long load_int(const void *p, int dt, long long i)
{
    switch (dt) {
    case TDP_I8: return ((const int8_t *)p)[i];
    case TDP_U8: return ((const uint8_t *)p)[i];
    case TDP_I32: return ((const int32_t *)p)[i];
    default: return ((const long long *)p)[i];
    }
}

// Loads 4 consecutive integer elements starting at row r (r % 4 == 0),
// widened to int64.  Rows >= n read as 0 (the caller masks them out).
__device__ __forceinline__ void load4_int(const void *p, int dt, bool vec_ok, long long r, long long n,
                                          long long v[4])
{
    if (vec_ok && r + 3 < n) {
        switch (dt) {
        case TDP_I8: {
            int w = __ldg((const int *)((const int8_t *)p + r));
            v[0] = (int8_t)(w & 0xff);
            v[1] = (int8_t)((w >> 8) & 0xff);
            v[2] = (int8_t)((w >> 16) & 0xff);
            v[3] = (int8_t)((w >> 24) & 0xff);
            return;
        }
        case TDP_U8: {
            unsigned w = __ldg((const unsigned *)((const uint8_t *)p + r));
            v[0] = w & 0xff;
            v[1] = (w >> 8) & 0xff;
            v[2] = (w >> 16) & 0xff;
            v[3] = (w >> 24) & 0xff;
            return;
        }
        case TDP_I32: {
            int4 w = __ldg((const int4 *)((const int32_t *)p + r));
            v[0] = w.x;
            v[1] = w.y;
            v[2] = w.z;
            v[3] = w.w;
            return;
        }
        default: {
            longlong2 a = __ldg((const longlong2 *)((const long long *)p + r));
            longlong2 b = __ldg((const longlong2 *)((const long long *)p + r + 2));
            v[0] = a.x;
            v[1] = a.y;
            v[2] = b.x;
            v[3] = b.y;
            return;
        }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
        v[k] = (r + k < n) ? load_int(p, dt, r + k) : 0;
}

// Range form of predicate p for a value already widened to 32 bits (I8, U8,
// I32 columns; lo/hi are clamped into the column type, so hi - lo fits).
__device__ __forceinline__ unsigned range_holds32(int v, int lo, unsigned span, unsigned neg)
{
    return ((unsigned)(v - lo) <= span ? 1u : 0u) ^ neg;
}

__device__ __forceinline__ unsigned range_holds64(long long v, long long lo, unsigned long long span, unsigned neg)
{
    return ((unsigned long long)(v - lo) <= span ? 1u : 0u) ^ neg;
}

__device__ __forceinline__ bool cmp_holds(long long v, int cmp, long long lit)
{
    switch (cmp) {
    case TDP_LT: return v < lit;
    case TDP_LE: return v <= lit;
    case TDP_GT: return v > lit;
    case TDP_GE: return v >= lit;
    case TDP_EQ: return v == lit;
    default: return v != lit;
    }
}

// 4-bit mask of rows r..r+3 (r % 4 == 0) that are < n and satisfy every predicate.
__device__ __forceinline__ unsigned eval_preds4(const PredSet &ps, long long r, long long n)
{
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        m |= (r + k < n) ? (1u << k) : 0u;
    for (int p = 0; p < ps.n; p++) {
        long long v[4];
        load4_int(ps.col[p], ps.dt[p], ps.vec_ok[p], r, n, v);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (!cmp_holds(v[k], ps.cmp[p], ps.lit[p]))
                m &= ~(1u << k);
    }
    return m;
}

// Same for a single row.
__device__ __forceinline__ bool eval_preds1(const PredSet &ps, long long r)
{
    for (int p = 0; p < ps.n; p++)
        if (!cmp_holds(load_int(ps.col[p], ps.dt[p], r), ps.cmp[p], ps.lit[p]))
            return false;
    return true;
}

// ------------------------------------------------ bulk copies and mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of bulk-copy data to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy (both addresses 16-byte aligned, bytes a
// multiple of 16) completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Shared -> global bulk copy (both addresses 16-byte aligned, bytes a
// multiple of 16), in the issuing thread's current bulk group.  The shared
// source must have been fenced for the async proxy by its writers.
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until at most N of the thread's bulk groups are still reading their
// shared source.
template <int N> __device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Waits until all of the thread's bulk groups have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// L2 cache policies: data read once (streamed columns, gathered columns) is
// marked evict-first so that it does not push out data read many times (a
// hash table), which is marked evict-last.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bulk_load with an L2 cache policy
__device__ __forceinline__ void bulk_load_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                               uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Read-only loads with an L2 cache policy.
__device__ __forceinline__ unsigned long long ldg_hint(const unsigned long long *p, uint64_t policy)
{
    unsigned long long v;
    asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(policy));
    return v;
}

__device__ __forceinline__ long long ldg_hint(const long long *p, uint64_t policy)
{
    long long v;
    asm("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(policy));
    return v;
}

__device__ __forceinline__ int32_t ldg_hint(const int32_t *p, uint64_t policy)
{
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
    return v;
}

__device__ __forceinline__ uint4 ldg16_hint(const uint32_t *p, uint64_t policy)
{
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(policy));
    return v;
}

// Plain mbarrier arrival (release at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the phase of the given parity; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done)
            return true;
    }
    return false;
}

// Bounded wait for an mbarrier phase that sleeps briefly between polls, so
// that warps whose stage is still in flight leave the issue slots to warps
// that have data.  False when the limit ran out.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done)
            return true;
        __nanosleep(64);
    }
    return false;
}

// Grid-wide barrier of a cooperative launch: every block adds one to the
// counter and waits (bounded) until all blocks of this round have.
__device__ __forceinline__ void grid_barrier(unsigned *counter, unsigned target, uint32_t limit, int32_t *d_status)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        uint32_t polls = 0;
        while (ld_relaxed_u32(counter) < target) {
            if (polls++ >= limit) {
                set_status(d_status, TDP_ERR_TIMEOUT);
                break;
            }
            __nanosleep(polls < 64 ? 32 : 256);
        }
        __threadfence();
    }
    __syncthreads();
}

// --------------------------------------------------------- decoupled look-back
//
// Tile status word: bits 62..63 flag (0 = nothing yet, 1 = tile aggregate,
// 2 = inclusive prefix), bits 0..61 the value.
constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_INC = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;

// True once any bounded wait of the call has timed out: later waits give up
// at once, so one stuck chain cannot make every tile wait its full limit.
__device__ __forceinline__ bool timed_out_already(const int32_t *d_status)
{
    return d_status && (*(volatile const int32_t *)d_status & TDP_ERR_TIMEOUT);
}

// Bounded spin on one status word until its flag is non-zero.  Gives up
// after `limit` polls (or when another wait already gave up), sets
// TDP_ERR_TIMEOUT and returns the word as read.
__device__ __forceinline__ unsigned long long lb_wait(const unsigned long long *w, uint32_t limit,
                                                      int32_t *d_status)
{
    unsigned long long s = ld_relaxed_u64(w);
    uint32_t polls = 0;
    while ((s >> 62) == 0) {
        if (polls++ >= limit || ((polls & 63) == 0 && timed_out_already(d_status))) {
            set_status(d_status, TDP_ERR_TIMEOUT);
            return s;
        }
        __nanosleep(polls < 64 ? 20 : 200);
        s = ld_relaxed_u64(w);
    }
    return s;
}

// Called by ONE full warp of the tile.  Publishes the tile aggregate, walks
// back over predecessors 32 at a time and returns the exclusive prefix
// (the same value in every lane); publishes the inclusive prefix.
__device__ __forceinline__ unsigned long long lookback_exclusive(unsigned long long *status, long long tile,
                                                                 unsigned long long aggregate, uint32_t limit,
                                                                 int32_t *d_status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0)
            st_relaxed_u64(&status[0], LB_INC | aggregate);
        return 0;
    }
    if (lane == 0)
        st_relaxed_u64(&status[tile], LB_AGG | aggregate);
    unsigned long long excl = 0;
    long long base = tile - 1;
    while (true) {
        long long t = base - lane;
        unsigned long long s = (t >= 0) ? lb_wait(&status[t], limit, d_status) : LB_INC;
        unsigned long long v = (t >= 0) ? (s & LB_VAL) : 0;
        unsigned incl_mask = __ballot_sync(0xffffffffu, (s >> 62) == 2 || (s >> 62) == 0);
        // (a timed-out predecessor is treated as an inclusive prefix of its value)
        int stop = incl_mask ? __ffs(incl_mask) - 1 : 32;
        unsigned long long contrib = (lane <= stop) ? v : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        excl += contrib;
        if (incl_mask)
            break;
        base -= 32;
    }
    if (lane == 0)
        st_relaxed_u64(&status[tile], LB_INC | ((excl + aggregate) & LB_VAL));
    return excl;
}

} // namespace tdp
