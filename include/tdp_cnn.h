/*
 * tdp_cnn.h -- C ABI of the trainable glyph query (B300, sm_103a).
 *
 * The paper's trainable query (Sec. 3 training loop; Sec. 4 soft operators on
 * probability-encoded (PE) columns; Sec. 5.5 queries over image grids) runs a
 * CNN over every cell of a grid image, turns the class probabilities (the PE
 * column, softmax as the proxy for argmax) into a soft per-class COUNT and a
 * soft per-row SUM of class values, and trains the CNN end to end with an MSE
 * loss against the same query run exactly on known labels, using Adam.  At
 * inference the exact query (argmax, integer COUNT/SUM) replaces the soft one.
 *
 * Network: conv3x3 1->32 + ReLU, conv3x3 32->64 + ReLU, maxpool 2x2,
 * FC 9216->128 + ReLU, FC 128->10, softmax.  Grids are 4x4 cells of 28x28.
 *
 * Tensors (all DEVICE memory owned by the caller; same conventions as tdp.h:
 * asynchronous on `stream`, no allocation, host status for argument errors):
 *   grids   uint8  [n_grids][112][112]   cell (r, c) is rows 28r.., cols 28c..
 *   y1      bf16   [n_cells][26][26][32] conv1 output after ReLU (NHWC)
 *   y2      bf16   [n_cells][12][12][64] pooled conv2 output after ReLU
 *   argmax  uint8  [n_cells][12][12][64] window position (dy*2+dx) of the max,
 *                                         first maximum on ties
 *   h1      bf16   [n_cells][128]        fc1 output after ReLU
 *   conv1 weights fp32 w1 [32][3][3], b1 [32]
 *   conv2 weights bf16 w2 [64][3][3][32] (out, ky, kx, in), fp32 b2 [64]
 *   fc1 weights   bf16 wfc1 [128][9216] (inputs in (y, x, c) order), fp32 bfc1
 *   fc2 weights   fp32 wfc2 [10][128], bfc2 [10]
 * n_cells = 16 * n_grids.  "bf16" buffers are passed as void*.
 */
#ifndef TDP_CNN_H
#define TDP_CNN_H

#include "tdp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* conv1 + bias + ReLU, reading the cells in place from the grid images
 * (the split of a grid into cells is index arithmetic, no copy): grids u8
 * [n_grids][112][112], w1 fp32 [32][3][3], b1 fp32 [32], y1 bf16
 * [n_grids*16][26][26][32] (16-byte aligned, else TDP_ERR_INVALID_ARG). */
tdp_status tdp_cnn_conv1_fwd(const uint8_t *grids, int64_t n_grids, const float *w1, const float *b1, void *y1,
                             tdp_stream_t stream);

/* conv2 + bias + ReLU + 2x2 max-pool as one implicit GEMM on the 5th-gen
 * tensor cores (tcgen05: bf16 operands staged in shared memory, fp32
 * accumulator in tensor memory); writes y2 and argmax.  y1, w2, y2 and argmax
 * must be 16-byte aligned (TDP_ERR_INVALID_ARG otherwise).  A bounded device
 * wait that runs out sets TDP_ERR_TIMEOUT in *d_status (nullable). */
tdp_status tdp_cnn_conv2_pool_fwd(const void *y1, int64_t n_cells, const void *w2, const float *b2, void *y2,
                                  uint8_t *argmax, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_fc1_fwd. */
size_t tdp_cnn_fc1_fwd_workspace(int64_t n_cells);

/*
 * fc1 + bias + ReLU: h1 bf16 [n_cells][128] = relu(y2 . wfc1^T + bfc1), y2 bf16
 * [n_cells][9216], wfc1 bf16 [128][9216], bfc1 fp32 [128].  A split-K GEMM on
 * the 5th-gen tensor cores (tcgen05), fp32 partials summed in ws in a fixed
 * order.  y2 and wfc1 must be 16-byte aligned, else TDP_ERR_INVALID_ARG.  A
 * bounded device wait that runs out sets TDP_ERR_TIMEOUT in *d_status
 * (nullable).
 */
tdp_status tdp_cnn_fc1_fwd(const void *y2, int64_t n_cells, const void *wfc1, const float *bfc1, void *h1, void *ws,
                           size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_head. */
size_t tdp_cnn_head_workspace(int64_t n_grids);

/*
 * fc2 + softmax + soft query, and (when targets != NULL) the loss and its
 * backward, one block per grid:
 *   logits [n_cells][10], P [n_cells][10]   (each optional)
 *   pred   [n_grids][14]  = 10 soft counts  cnt[k]  = sum_cells P[c][k]
 *                         + 4 soft row sums rsum[r] = sum_{c in row r} sum_k k P[c][k]
 *   with targets [n_grids][14] (the exact query on true labels):
 *   loss   [1]  = mean over the n_grids x 14 outputs of (pred - target)^2
 *   dh1    bf16 [n_cells][128]  gradient of the MSE mean w.r.t. h1 (ReLU-masked)
 *   dwfc2  [10][128], dbfc2 [10]  its fc2 gradients (per-grid partials in ws,
 *                                 summed in grid order in float64)
 */
tdp_status tdp_cnn_head(const void *h1, int64_t n_grids, const float *wfc2, const float *bfc2, const float *targets,
                        float *logits, float *P, float *pred, void *dh1, float *dwfc2, float *dbfc2, float *loss,
                        void *ws, size_t ws_bytes, tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_head2. */
size_t tdp_cnn_head2_workspace(int64_t n_grids);

/*
 * Head of the two-attribute query (Digit x Size, Sec. 4 soft group-by over
 * two PE columns of the same cells), one block per grid: the digit head
 * wfc2 [10][128], bfc2 [10] and the size head wfc2s [2][128], bfc2s [2], both
 * on h1, one softmax each, and the soft COUNT of every (digit, size) pair
 *   pred [n_grids][10][2], pred[g][a][b] = sum_cells P[c][a] * Ps[c][b]
 * logits [n_cells][10], logits_s [n_cells][2], P [n_cells][10], Ps
 * [n_cells][2] are optional outputs.  With targets [n_grids][10][2] (the exact
 * pair counts on true labels): loss [1] = mean of the 20 n_grids squared
 * errors, dh1 bf16 [n_cells][128] (both heads' gradients added, ReLU-masked),
 * dwfc2, dbfc2, dwfc2s, dbfc2s (per-grid partials in ws summed in grid order
 * in float64).  Argument errors as tdp_cnn_head.
 */
tdp_status tdp_cnn_head2(const void *h1, int64_t n_grids, const float *wfc2, const float *bfc2, const float *wfc2s,
                         const float *bfc2s, const float *targets, float *logits, float *logits_s, float *P,
                         float *Ps, float *pred, void *dh1, float *dwfc2, float *dbfc2, float *dwfc2s,
                         float *dbfc2s, float *loss, void *ws, size_t ws_bytes, tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_fc1_bwd. */
size_t tdp_cnn_fc1_bwd_workspace(int64_t n_cells);

/*
 * fc1 backward from dh1 bf16 [n_cells][128] (the gradient at fc1's output,
 * ReLU applied).  dy2p bf16 [n_cells][9216] = (dh1 . wfc1) masked by y2 > 0
 * (the gradient at the pooled map, through the ReLU); dwfc1 fp32 [128][9216]
 * = dh1^T . y2 (split-K); dbfc1 fp32 [128] = column sums of dh1.  Both
 * products on the 5th-gen tensor cores (tcgen05).  dh1, y2, wfc1 and dy2p
 * must be 16-byte aligned, else TDP_ERR_INVALID_ARG.  A bounded device wait
 * that runs out sets TDP_ERR_TIMEOUT in *d_status (nullable).
 */
tdp_status tdp_cnn_fc1_bwd(const void *dh1, const void *y2, const void *wfc1, int64_t n_cells, void *dy2p,
                           float *dwfc1, float *dbfc1, void *ws, size_t ws_bytes, int32_t *d_status,
                           tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_conv2_bwd. */
size_t tdp_cnn_conv2_bwd_workspace(int64_t n_cells);

/*
 * conv2 backward from the pooled gradient dy2p and the pool arg-max: the
 * gradient at each conv2 output pixel is the pooled gradient where that pixel
 * is its window's arg-max, else 0 (expanded on the fly, never stored).
 *   dz1 bf16 [n_cells][26][26][32] = (conv2 transposed) masked by y1 > 0
 *       (optional: NULL skips the data gradient)
 *   dw2 fp32 [64][3][3][32], db2 fp32 [64]
 * The data gradient runs on the 5th-gen tensor cores (tcgen05, nine
 * accumulating GEMMs over shifted views of one gradient patch); dy2p,
 * argmax, y1 and dz1 must be 16-byte aligned.  A bounded device wait that
 * runs out sets TDP_ERR_TIMEOUT in *d_status (nullable).
 */
tdp_status tdp_cnn_conv2_bwd(const void *dy2p, const uint8_t *argmax, const void *y1, const void *w2, int64_t n_cells,
                             void *dz1, float *dw2, float *db2, void *ws, size_t ws_bytes, int32_t *d_status,
                             tdp_stream_t stream);

/* Workspace bytes of tdp_cnn_conv1_bwd. */
size_t tdp_cnn_conv1_bwd_workspace(int64_t n_cells);

/*
 * conv1 weight and bias gradients from dz1 bf16 [n_cells][26][26][32] (the
 * gradient at conv1's output, ReLU applied): dw1 fp32 [32][3][3] (the
 * correlation of dz1 with the cell image / 255), db1 fp32 [32] (the sum of
 * dz1 per channel).  dz1 must be 4-byte aligned, n_cells a multiple of 16
 * (whole grids), else TDP_ERR_INVALID_ARG.  Deterministic for a given GPU.
 */
tdp_status tdp_cnn_conv1_bwd(const void *dz1, const uint8_t *grids, int64_t n_cells, float *dw1, float *db1, void *ws,
                             size_t ws_bytes, tdp_stream_t stream);

/*
 * One Adam step (the optimiser of the paper's training loop) over up to 16
 * fp32 tensors: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * bf16_copies[i] (optional, or NULL entries) receives p rounded to bf16, the
 * operand copy the tensor-core layers read.  step >= 1.
 */
tdp_status tdp_adam_step(float *const *params, const float *const *grads, float *const *m, float *const *v,
                         void *const *bf16_copies, const int64_t *sizes, int32_t count, int32_t step, float lr,
                         float beta1, float beta2, float eps, tdp_stream_t stream);

/* y[i] = bf16(x[i]) (round to nearest even). */
tdp_status tdp_f32_to_bf16(const float *x, int64_t n, void *y, tdp_stream_t stream);

/*
 * Exact query at inference (Sec. 4: exact operators replace the soft ones):
 * per cell the first arg-max of its K logits (labels [n_grids*gh*gw], optional),
 * per grid the exact integer COUNT per class cnt [n_grids][K] and the per-row
 * SUM of class values rsum [n_grids][gh].
 */
tdp_status tdp_exact_pe_count(const float *logits, int64_t n_grids, int32_t K, int32_t grid_h, int32_t grid_w,
                              int32_t *labels, int64_t *cnt, int64_t *rsum, tdp_stream_t stream);

/*
 * Soft group-by on a PE column (Sec. 4 soft_count / soft_groupby; only + and
 * x): P [n_grids*gh*gw][K] (cells of a grid row-major), cnt [n_grids][K],
 * rsum [n_grids][gh] as in tdp_cnn_head.  The backward is the adjoint:
 * dP[c][k] = dcnt[g][k] + k * drsum[g][row(c)].
 */
tdp_status tdp_pe_groupby_fwd(const float *P, int64_t n_grids, int32_t K, int32_t grid_h, int32_t grid_w, float *cnt,
                              float *rsum, tdp_stream_t stream);
tdp_status tdp_pe_groupby_bwd(const float *dcnt, const float *drsum, int64_t n_grids, int32_t K, int32_t grid_h,
                              int32_t grid_w, float *dP, tdp_stream_t stream);

/*
 * Exact pair query at inference: per cell the first arg-max of logits_a
 * [n_grids*cells][Ka] and of logits_b [n_grids*cells][Kb] (labels_a,
 * labels_b [n_grids*cells], each optional), per grid the integer COUNT of
 * every pair, cnt [n_grids][Ka][Kb].
 */
tdp_status tdp_exact_pe_count2(const float *logits_a, int32_t Ka, const float *logits_b, int32_t Kb, int64_t n_grids,
                               int32_t cells, int32_t *labels_a, int32_t *labels_b, int64_t *cnt,
                               tdp_stream_t stream);

/*
 * Soft pair COUNT over two PE columns of the same cells (Sec. 4 soft
 * group-by on two attributes): cnt [n_grids][Ka][Kb] = sum over the grid's
 * `cells` consecutive cells of Pa[c][a] * Pb[c][b].  The backward is the
 * adjoint of this bilinear map: dPa[c][a] = sum_b dcnt[g][a][b] Pb[c][b],
 * dPb[c][b] = sum_a dcnt[g][a][b] Pa[c][a].
 */
tdp_status tdp_pe_groupby2_fwd(const float *Pa, int32_t Ka, const float *Pb, int32_t Kb, int64_t n_grids,
                               int32_t cells, float *cnt, tdp_stream_t stream);
tdp_status tdp_pe_groupby2_bwd(const float *dcnt, const float *Pa, int32_t Ka, const float *Pb, int32_t Kb,
                               int64_t n_grids, int32_t cells, float *dPa, float *dPb, tdp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TDP_CNN_H */
