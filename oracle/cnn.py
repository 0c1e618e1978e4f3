"""fp64 oracle for the trainable glyph query (Sec. 3 training loop, Sec. 4,
Sec. 5.5 query over image grids).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The query: a grid image is split into 4x4 cells; a CNN maps each 28x28 cell
to class probabilities (softmax, the PE column); the soft group-by turns the
probabilities of the 16 cells into a per-class COUNT and a per-row SUM of
class values; the loss is the mean squared error against the same query run
exactly on the true labels; training backpropagates through the query into
the CNN and takes Adam steps (lr 0.01 in the paper's loop).

Network (one reading of the paper's unspecified ``CNN(num_classes=10)``):
  conv3x3(1->32, valid) + ReLU -> conv3x3(32->64, valid) + ReLU
  -> maxpool 2x2 -> flatten (y, x, c) -> FC 9216->128 + ReLU -> FC 128->10
  -> softmax.

``quant=True`` reproduces the precision contract of the accelerated path in
float64 arithmetic: the conv2 / fc1 operands (activations and weights) and
the back-propagated activation gradients that feed those contractions are
rounded to bfloat16 (round to nearest even) at the same points, everything
else stays float64.  ``quant=False`` is the plain float64 network used for
the finite-difference pins.

Direct-loop formulation: each 3x3 convolution is a sum over the 9 kernel
taps of shifted-window contractions (numpy ``@`` / ``einsum`` as the
library step); pooling takes the first maximal element of each 2x2 window in
(dy, dx) row-major order.
"""
from __future__ import annotations

import numpy as np

from . import soft

K_CLASSES = 10
GRID = 4
CELL = 28


def bf16(a):
    """Round float values to the nearest bfloat16 (ties to even); float64 out."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def split_cells(grids_u8):
    """[n, 112, 112] grid images -> [n*16, 28, 28] cells (row-major cells)."""
    g = np.asarray(grids_u8)
    n = g.shape[0]
    return g.reshape(n, GRID, CELL, GRID, CELL).transpose(0, 1, 3, 2, 4).reshape(n * GRID * GRID, CELL, CELL)


def _q(a, quant):
    return bf16(a) if quant else np.asarray(a, np.float64)


def conv1_relu(x0, w1, b1):
    """conv3x3 (1 -> 32, valid) + bias + ReLU; x0 [B,28,28] -> [B,26,26,32]."""
    B = x0.shape[0]
    z1 = np.zeros((B, 26, 26, 32))
    for ky in range(3):
        for kx in range(3):
            z1 += x0[:, ky:ky + 26, kx:kx + 26, None] * w1[:, ky, kx]
    z1 += b1
    return np.maximum(z1, 0.0)


def conv2_relu_pool(y1, w2, b2):
    """conv3x3 (32 -> 64, valid) + bias + ReLU, then 2x2 max-pool taking the
    first maximum of each window in (dy, dx) order.  Returns (pooled
    [B,12,12,64], argmax window position [B,12,12,64], a2 [B,24,24,64])."""
    B = y1.shape[0]
    z2 = np.zeros((B, 24, 24, 64))
    for ky in range(3):
        for kx in range(3):
            z2 += y1[:, ky:ky + 24, kx:kx + 24, :] @ w2[:, ky, kx, :].T
    z2 += b2
    a2 = np.maximum(z2, 0.0)
    win = a2.reshape(B, 12, 2, 12, 2, 64).transpose(0, 1, 3, 2, 4, 5).reshape(B, 12, 12, 4, 64)
    arg = np.argmax(win, axis=3)  # first occurrence of the maximum
    pooled = np.take_along_axis(win, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :]
    return pooled, arg, a2


def conv2_backward(dy2, arg, y1, w2):
    """Backward of conv2 + ReLU + 2x2 max-pool from the pooled gradient dy2
    [B,12,12,64] (already masked by the pooled ReLU) and the pool arg-max:
    the pre-pool gradient dz2 is dy2 at each window's arg-max pixel and 0
    elsewhere.  Returns (dz1 [B,26,26,32] = the transposed convolution of
    dz2 masked by y1 > 0, dw2 [64,3,3,32], db2 [64]).  float64."""
    B = dy2.shape[0]
    dwin = np.zeros((B, 12, 12, 4, 64))
    np.put_along_axis(dwin, np.asarray(arg)[:, :, :, None, :], np.asarray(dy2, np.float64)[:, :, :, None, :], axis=3)
    dz2 = dwin.reshape(B, 12, 12, 2, 2, 64).transpose(0, 1, 3, 2, 4, 5).reshape(B, 24, 24, 64)
    y1 = np.asarray(y1, np.float64)
    w2 = np.asarray(w2, np.float64)
    gw2 = np.zeros((64, 3, 3, 32))
    dy1 = np.zeros((B, 26, 26, 32))
    for ky in range(3):
        for kx in range(3):
            gw2[:, ky, kx, :] = np.einsum("byxo,byxi->oi", dz2, y1[:, ky:ky + 24, kx:kx + 24, :])
            dy1[:, ky:ky + 24, kx:kx + 24, :] += dz2 @ w2[:, ky, kx, :]
    return dy1 * (y1 > 0), gw2, dz2.sum(axis=(0, 1, 2))


def fc1_backward(dh1, flat, wf1):
    """fc1 gradients from dh1 [B, 128] (the gradient at fc1's output, ReLU
    applied), its input flat [B, 9216] (the pooled map, itself a ReLU output)
    and weights wf1 [128, 9216]: (dh1 . wf1 masked by flat > 0, the gradient
    at the pooled map through its ReLU; dW = dh1^T . flat; db = column sums of
    dh1).  float64."""
    dh1 = np.asarray(dh1, np.float64)
    flat = np.asarray(flat, np.float64)
    return (dh1 @ np.asarray(wf1, np.float64)) * (flat > 0), dh1.T @ flat, dh1.sum(axis=0)


def conv1_backward(dz1, x0):
    """conv1 weight and bias gradients of the valid 3x3 correlation in the
    Sec. 5.5 CNN: dW1[o, ky, kx] = sum over cells
    and output pixels of dz1[b, y, x, o] * x0[b, y+ky, x+kx]; db1[o] = sum of
    dz1[..., o].  dz1 [B, 26, 26, 32], x0 [B, 28, 28] (pixels / 255)."""
    dz1 = np.asarray(dz1, np.float64)
    x0 = np.asarray(x0, np.float64)
    gw1 = np.zeros((32, 3, 3))
    for ky in range(3):
        for kx in range(3):
            gw1[:, ky, kx] = np.einsum("byxo,byx->o", dz1, x0[:, ky:ky + 26, kx:kx + 26])
    return gw1, dz1.sum(axis=(0, 1, 2))


def fc(x, w, b, relu):
    z = x @ w.T + b
    return np.maximum(z, 0.0) if relu else z


def forward(params, grids_u8, quant=True):
    """Returns a dict with every intermediate needed by ``backward``."""
    p = {k: np.asarray(v, np.float64) for k, v in params.items()}
    x0 = split_cells(grids_u8).astype(np.float64) / 255.0  # [B,28,28]
    B = x0.shape[0]
    y1 = _q(conv1_relu(x0, p["conv1_w"], p["conv1_b"]), quant)
    w2 = _q(p["conv2_w"], quant)
    pooled, arg, a2 = conv2_relu_pool(y1, w2, p["conv2_b"])
    y2 = _q(pooled, quant)  # [B,12,12,64]
    flat = y2.reshape(B, 9216)
    wf1 = _q(p["fc1_w"], quant)
    h1 = _q(fc(flat, wf1, p["fc1_b"], True), quant)
    logits = fc(h1, p["fc2_w"], p["fc2_b"], False)
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    P = e / e.sum(axis=1, keepdims=True)
    cnt, rsum = soft.pe_groupby_fwd(P)
    pred = np.concatenate([cnt, rsum], axis=1)  # [n_grids, 14]
    return dict(x0=x0, y1=y1, w2=w2, a2=a2, arg=arg, y2=y2, wf1=wf1, h1=h1,
                logits=logits, P=P, pred=pred, quant=quant)


def targets_from_labels(labels):
    """Exact query on the true labels: [n_grids, 14] (10 counts, 4 row sums)."""
    cnt, rsum = soft.exact_groupby(labels, K_CLASSES)
    return np.concatenate([cnt, rsum], axis=1).astype(np.float64)


def loss(pred, target):
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d))


def _trunk_backward(p, fw, dh1, quant):
    """Gradients of fc1, conv2 and conv1 from the hidden-layer gradient dh1
    (ReLU applied, rounded as the accelerated path rounds it)."""
    g = {}
    B = dh1.shape[0]
    flat = fw["y2"].reshape(B, 9216)
    dflat, g["fc1_w"], g["fc1_b"] = fc1_backward(dh1, flat, fw["wf1"])
    dy2 = _q(dflat.reshape(B, 12, 12, 64), quant)
    dz1, g["conv2_w"], g["conv2_b"] = conv2_backward(dy2, fw["arg"], fw["y1"], fw["w2"])
    dz1 = _q(dz1, quant)
    g["conv1_w"], g["conv1_b"] = conv1_backward(dz1, fw["x0"])
    return g


def backward(params, fw, target):
    """Gradients of the MSE loss w.r.t. every parameter (dict like params)."""
    p = {k: np.asarray(v, np.float64) for k, v in params.items()}
    quant = fw["quant"]
    pred = fw["pred"]
    n_out = pred.size
    dpred = 2.0 * (pred - np.asarray(target, np.float64)) / n_out
    dP = soft.pe_groupby_bwd(dpred[:, :K_CLASSES], dpred[:, K_CLASSES:])
    P = fw["P"]
    dlogits = P * (dP - (P * dP).sum(axis=1, keepdims=True))
    h1 = fw["h1"]
    g = {}
    g["fc2_w"] = dlogits.T @ h1
    g["fc2_b"] = dlogits.sum(axis=0)
    dh1 = _q((dlogits @ p["fc2_w"]) * (h1 > 0), quant)
    g.update(_trunk_backward(p, fw, dh1, quant))
    return g


def adam_step(params, grads, m, v, t, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments), float64.  Returns new
    (params, m, v)."""
    newp, newm, newv = {}, {}, {}
    for k in params:
        gk = np.asarray(grads[k], np.float64)
        mk = b1 * np.asarray(m[k], np.float64) + (1 - b1) * gk
        vk = b2 * np.asarray(v[k], np.float64) + (1 - b2) * gk * gk
        mhat = mk / (1 - b1 ** t)
        vhat = vk / (1 - b2 ** t)
        newp[k] = np.asarray(params[k], np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
        newm[k], newv[k] = mk, vk
    return newp, newm, newv


def predict_labels(params, grids_u8):
    """Exact-mode inference: argmax of the class probabilities per cell."""
    fw = forward(params, grids_u8, quant=False)
    return np.argmax(fw["logits"], axis=1).reshape(-1, GRID, GRID)


# ------------------------------------------- two heads: Digit x Size query

K_SIZES = 2


def _softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def forward2(params, size_params, grids_u8, quant=True):
    """The Digit x Size query: the digit head (fc2) and a size head (fc2s,
    128 -> 2) on the same hidden layer, one softmax each, then
    cnt[d, s] = sum_c P_digit[c, d] P_size[c, s] per grid (20 outputs)."""
    fw = forward(params, grids_u8, quant)
    q = {k: np.asarray(v, np.float64) for k, v in size_params.items()}
    ls = fc(fw["h1"], q["fc2s_w"], q["fc2s_b"], False)
    Ps = _softmax(ls)
    cnt = soft.pe_groupby2_fwd(fw["P"], Ps)
    fw2 = dict(fw)
    fw2.update(logits_s=ls, Ps=Ps, pred2=cnt.reshape(cnt.shape[0], -1))
    return fw2


def targets2(digits, sizes):
    """Exact Digit x Size counts on the true labels: [n_grids, 20]."""
    c = soft.exact_groupby2(digits, sizes, K_CLASSES, K_SIZES)
    return c.reshape(c.shape[0], -1).astype(np.float64)


def backward2(params, size_params, fw2, target):
    """Gradients of the MSE of the 20 Digit x Size counts w.r.t. every
    parameter of both heads and the shared trunk."""
    p = {k: np.asarray(v, np.float64) for k, v in params.items()}
    q = {k: np.asarray(v, np.float64) for k, v in size_params.items()}
    quant = fw2["quant"]
    pred = fw2["pred2"]
    dpred = 2.0 * (pred - np.asarray(target, np.float64)) / pred.size
    dPd, dPs = soft.pe_groupby2_bwd(dpred.reshape(-1, K_CLASSES, K_SIZES), fw2["P"], fw2["Ps"])
    P, Ps, h1 = fw2["P"], fw2["Ps"], fw2["h1"]
    dld = P * (dPd - (P * dPd).sum(axis=1, keepdims=True))
    dls = Ps * (dPs - (Ps * dPs).sum(axis=1, keepdims=True))
    g = {"fc2_w": dld.T @ h1, "fc2_b": dld.sum(axis=0), "fc2s_w": dls.T @ h1, "fc2s_b": dls.sum(axis=0)}
    dh1 = _q((dld @ p["fc2_w"] + dls @ q["fc2s_w"]) * (h1 > 0), quant)
    g.update(_trunk_backward(p, fw2, dh1, quant))
    return g


def predict_labels2(params, size_params, grids_u8):
    """Exact mode: argmax of each head per cell -> (digits, sizes) [n, 4, 4]."""
    fw2 = forward2(params, size_params, grids_u8, quant=False)
    n = np.asarray(grids_u8).shape[0]
    return (np.argmax(fw2["logits"], axis=1).reshape(n, GRID, GRID),
            np.argmax(fw2["logits_s"], axis=1).reshape(n, GRID, GRID))
