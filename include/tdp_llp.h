/*
 * tdp_llp.h -- C ABI of learning from label proportions (B300, sm_103a).
 *
 * Sec. 5.3 trains a linear classifier (a table-valued function) from bags of
 * rows that carry only a per-bag COUNT of each class: the query
 * SELECT class, COUNT(*) ... GROUP BY class runs softly on every bag (softmax
 * in place of argmax, Sec. 4), so a bag's soft count of class k is the sum of
 * its rows' probabilities of k, and the mean squared error between the soft
 * counts and the bags' count labels is minimised (with tdp_adam_step,
 * tdp_cnn.h).  Sec. 5.4 trains on the same counts after the Laplace
 * mechanism (label differential privacy).
 *
 *   bag j          rows j*B .. min(n, (j+1)*B) - 1   (the last bag may be short)
 *   P[i][k]        softmax_k(sum_f X[i][f] W[k][f] + b[k])
 *   cnt[j][k]      sum over the rows i of bag j of P[i][k]
 *   loss           mean over the n_bags x K counts of (cnt - target)^2
 *
 * Conventions as tdp.h: DEVICE pointers owned by the caller, asynchronous on
 * `stream`, no allocation, argument errors returned before any launch,
 * device-side conditions OR-ed into the caller-zeroed *d_status.  Shapes:
 * X fp32 [n][d] row-major, W fp32 [K][d], b fp32 [K], counts and targets
 * fp32 [n_bags][K] with n_bags = ceil(n / B).  Supported: 2 <= K <= 4,
 * 1 <= d <= 16, B >= 1, n >= 0 (n = 0: nothing launched, outputs untouched).
 */
#ifndef TDP_LLP_H
#define TDP_LLP_H

#include "tdp.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Count labels of the bags (the exact GROUP BY class COUNT per bag), with
 * the Laplace mechanism when noise != NULL:
 *   counts[j][k] = #{ i in bag j : labels[i] == k } + scale * noise[j][k]
 * labels int32 [n]; noise fp32 [n_bags][K] holds standard Laplace draws
 * (location 0, scale 1), drawn by the caller; scale = sensitivity / epsilon
 * (2 / 0.1 = 20 for the paper's epsilon, the count vector's L1 sensitivity
 * being 2).  A label outside [0, K) is not counted and sets
 * TDP_ERR_OVERFLOW in *d_status (nullable).  1 <= K <= 16 here.
 */
tdp_status tdp_llp_counts(const int32_t *labels, int64_t n, int32_t K, int64_t B, const float *noise, float scale,
                          float *counts, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes of tdp_llp_step (per-block partials). */
size_t tdp_llp_step_workspace(int64_t n, int32_t d, int32_t K, int64_t B);

/*
 * One forward + backward pass of the LLP query over all n rows, reading X
 * once from HBM: per bag the soft counts (written to cnt when not NULL),
 * the loss against targets [n_bags][K] into loss [1], and the gradients
 * dW [K][d], db [K] of that mean.  Bags never straddle a block's group of
 * rows (groups hold whole bags; a bag longer than one staged chunk is read
 * twice), so each bag's count gradient is formed where its rows are.  Sums
 * are per-block fp32 partials added in float64 in a fixed order, so results
 * are deterministic for a given GPU.  X must be 4-byte aligned.  With two
 * classes, at most 8 features and X 16-byte aligned, the rows stream
 * through shared memory by bulk copies; a bounded wait for one that runs out
 * sets TDP_ERR_TIMEOUT in *d_status (nullable) and the outputs are then
 * undefined.
 */
tdp_status tdp_llp_step(const float *X, int64_t n, int32_t d, int32_t K, int64_t B, const float *W, const float *b,
                        const float *targets, float *cnt, float *loss, float *dW, float *db, void *ws,
                        size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/*
 * The hard classifier at inference: labels_out[i] = first arg-max over k of
 * the logits (optional), and with ref_labels != NULL the number of rows whose
 * prediction differs from ref_labels[i], ADDED to *d_errors (int64, the
 * caller zeroes it).
 */
tdp_status tdp_llp_predict(const float *X, int64_t n, int32_t d, int32_t K, const float *W, const float *b,
                           int32_t *labels_out, const int32_t *ref_labels, int64_t *d_errors, tdp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TDP_LLP_H */
