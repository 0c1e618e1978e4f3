/*
 * tdp_softsort.h -- C ABI of a soft ORDER BY ... LIMIT k (B300, sm_103a).
 *
 * Sec. 4 makes discrete operators trainable by relaxing them, a logistic
 * function standing in for the step function of a comparison.  The paper
 * names sorting among the operators that can be relaxed so but fixes no
 * formula; these calls relax every comparison of a rank the way the soft
 * filter relaxes its predicate:
 *
 *   rank (descending, 1-based) of row i in its group g:
 *       r_i = 1 + sum_{j in g, j != i} sigma((x_j - x_i) / tau)
 *   top-k membership:  m_i = sigma((k + 1/2 - r_i) / tau_r)
 *   soft top-k sum:    S_g = sum_{i in g} m_i v_i
 *
 * and the exact operator (at inference) ranks by x descending with ties by
 * position and keeps the rows of rank <= k.
 *
 * Groups are runs of consecutive rows: rows offsets[g] .. offsets[g+1] - 1,
 * offsets int64 [n_groups + 1], offsets[0] = 0, offsets[n_groups] = n.  Each
 * group has at most max_group rows (the launch is sized by it): a group
 * with more rows, or with offsets out of order or out of [0, n], is skipped
 * and sets TDP_ERR_CAPACITY in *d_status (nullable).  The cost is
 * sum over groups of (group rows)^2 logistic evaluations.
 *
 * Conventions as tdp.h: DEVICE pointers owned by the caller, asynchronous
 * on `stream`, no allocation, argument errors returned before any launch.
 * x, v, rank, mask, dx, dv are fp32 [n]; sums are per group.  tau > 0,
 * tau_r > 0, k >= 1, 1 <= max_group <= 2^24.
 */
#ifndef TDP_SOFTSORT_H
#define TDP_SOFTSORT_H

#include "tdp.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Forward: rank [n] and mask [n] (both required; the backward reads mask),
 * and, when v and sum are given, sum fp32 [n_groups] = S_g (each group's
 * rows added in float64 in a fixed order, so deterministic).  Each rank sums
 * fp32 partials of 32 logistic terms with Kahan compensation.
 */
tdp_status tdp_soft_topk_fwd(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                             int64_t max_group, int32_t k, float tau, float tau_r, float *rank, float *mask,
                             float *sum, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes of tdp_soft_topk_bwd (the rank gradient, n floats). */
size_t tdp_soft_topk_workspace(int64_t n);

/*
 * Backward from upstream gradients dsum [n_groups], dmask [n], drank [n]
 * (each optional) and the forward's mask: dx [n] (required) and, when v and
 * dsum are given, dv [n] = dsum[g] * m_i (optional).  With
 * s_ij = sigma'((x_j - x_i) / tau) / tau:
 *   dm_i = dsum[g] v_i + dmask_i,  dr_i = -dm_i m_i (1 - m_i) / tau_r + drank_i,
 *   dx_i = sum_{j in g} s_ij (dr_j - dr_i).
 */
tdp_status tdp_soft_topk_bwd(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                             int64_t max_group, int32_t k, float tau, float tau_r, const float *mask,
                             const float *dsum, const float *dmask, const float *drank, float *dx, float *dv,
                             void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/*
 * The exact operator: rank int32 [n] = 1 + #{j in g : x_j > x_i, or
 * x_j == x_i and j < i} (required) and, when v and sum are given, sum
 * float64 [n_groups] = the SUM of v over the group's rows of rank <= k,
 * added in a fixed order.
 */
tdp_status tdp_exact_topk(const float *x, const float *v, int64_t n, const int64_t *offsets, int64_t n_groups,
                          int64_t max_group, int32_t k, int32_t *rank, double *sum, int32_t *d_status,
                          tdp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TDP_SOFTSORT_H */
