// Status strings, the bounded-wait knob and shared host helpers.
#include <atomic>

#include "common.cuh"

namespace tdp {

static std::atomic<uint32_t> g_spin_limit{1u << 20};

uint32_t spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }

int num_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

// The range [lo, hi] (and negation) equivalent to `v cmp lit` for values of
// type dt: LT/LE/GT/GE bound one side, EQ is [lit, lit], NE its complement.
// Bounds are clamped to the type's range; an empty range becomes the full
// range with neg = 1 (never true).
void pred_range(int dt, int cmp, long long lit, long long *lo, long long *hi, int32_t *neg)
{
    long long tmin, tmax;
    switch (dt) {
    case TDP_I8: tmin = -128, tmax = 127; break;
    case TDP_U8: tmin = 0, tmax = 255; break;
    case TDP_I32: tmin = INT32_MIN, tmax = INT32_MAX; break;
    default: tmin = INT64_MIN, tmax = INT64_MAX; break;
    }
    long long a = tmin, b = tmax;
    bool empty = false;
    int ng = 0;
    switch (cmp) {
    case TDP_LT:
        if (lit <= tmin) empty = true;
        else b = lit - 1 < tmax ? lit - 1 : tmax;
        break;
    case TDP_LE:
        if (lit < tmin) empty = true;
        else b = lit < tmax ? lit : tmax;
        break;
    case TDP_GT:
        if (lit >= tmax) empty = true;
        else a = lit + 1 > tmin ? lit + 1 : tmin;
        break;
    case TDP_GE:
        if (lit > tmax) empty = true;
        else a = lit > tmin ? lit : tmin;
        break;
    case TDP_EQ:
        if (lit < tmin || lit > tmax) empty = true;
        else a = b = lit;
        break;
    default: // NE
        if (lit < tmin || lit > tmax) {
            a = tmin, b = tmax; // always true
        } else {
            a = b = lit;
            ng = 1;
        }
        break;
    }
    if (empty) {
        a = tmin, b = tmax;
        ng = 1;
    }
    *lo = a;
    *hi = b;
    *neg = ng;
}

tdp_status make_predset(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds, int64_t n,
                        PredSet *out)
{
    if (npreds < 0 || npreds > TDP_MAX_PREDS || (npreds > 0 && (!preds || !cols)))
        return TDP_ERR_INVALID_ARG;
    out->n = npreds;
    for (int i = 0; i < npreds; i++) {
        int c = preds[i].col;
        if (c < 0 || c >= ncols || preds[i].cmp < TDP_LT || preds[i].cmp > TDP_NE)
            return TDP_ERR_INVALID_ARG;
        if (!is_int_dtype(cols[c].dtype))
            return TDP_ERR_UNSUPPORTED_DTYPE;
        if (cols[c].n < n || (n > 0 && !cols[c].data))
            return TDP_ERR_INVALID_ARG;
        out->col[i] = cols[c].data;
        out->dt[i] = cols[c].dtype;
        out->cmp[i] = preds[i].cmp;
        out->lit[i] = preds[i].lit;
        out->vec_ok[i] = ((uintptr_t)cols[c].data % 16) == 0;
        pred_range(cols[c].dtype, preds[i].cmp, preds[i].lit, &out->lo[i], &out->hi[i], &out->neg[i]);
    }
    for (int i = npreds; i < TDP_MAX_PREDS; i++) {
        out->col[i] = nullptr;
        out->dt[i] = 0;
        out->cmp[i] = 0;
        out->lit[i] = 0;
        out->vec_ok[i] = 0;
        out->lo[i] = 0;
        out->hi[i] = 0;
        out->neg[i] = 0;
    }
    return TDP_OK;
}

__global__ void debug_wait_kernel(const int32_t *flag, uint32_t polls, int32_t *d_status)
{
    if (threadIdx.x != 0)
        return;
    uint32_t i = 0;
    while (*(volatile const int32_t *)flag == 0) {
        if (i++ >= polls) {
            set_status(d_status, TDP_ERR_TIMEOUT);
            return;
        }
        __nanosleep(100);
    }
}

} // namespace tdp

extern "C" {

const char *tdp_status_str(int32_t s)
{
    switch (s) {
    case TDP_OK: return "ok";
    case TDP_ERR_INVALID_ARG: return "invalid argument";
    case TDP_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
    case TDP_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case TDP_ERR_CAPACITY: return "capacity exceeded";
    case TDP_ERR_DUP_BUILD_KEY: return "duplicate build key";
    case TDP_ERR_TIMEOUT: return "bounded device wait timed out";
    case TDP_ERR_OVERFLOW: return "arithmetic overflow";
    case TDP_ERR_CUDA: return "CUDA launch error";
    default: return "multiple device errors (bitwise OR of codes)";
    }
}

int32_t tdp_abi_version(void) { return 103; }

uint32_t tdp_set_spin_limit(uint32_t polls) { return tdp::g_spin_limit.exchange(polls); }

tdp_status tdp_debug_wait_flag(const int32_t *d_flag, uint32_t polls, int32_t *d_status, tdp_stream_t stream)
{
    if (!d_flag || !d_status)
        return TDP_ERR_INVALID_ARG;
    tdp::debug_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_flag, polls, d_status);
    return tdp::launch_status();
}

} // extern "C"
