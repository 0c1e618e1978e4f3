"""fp64 oracle for the differentiable ("trainable") query operators, Sec. 4.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4 relaxes discrete operators into differentiable ones: a logistic
function stands in for the step function of a filter predicate, softmax
stands in for argmax, and COUNT over probability-encoded (PE) columns is
built from additions and multiplications only; ``soft_groupby`` extends that
to grouped aggregation, and at inference the exact operators replace the soft
ones.  The formulas below are the plain definitions, evaluated in float64 on
the fp32 inputs widened to float64:

  soft filter      m_i = sigma((x_i - theta[g_i]) / tau)
  soft aggregation S[g] = sum_{g_i = g} v_i m_i ,  C[g] = sum_{g_i = g} m_i
  adjoints         dm_i/dtheta[g_i] = -m_i (1 - m_i) / tau ,
                   dm_i/dx_i = m_i (1 - m_i) / tau ,  dS/dv_i = m_i
  PE soft group-by cnt[n, k]  = sum_{cells c of grid n} P[c, k]
                   rsum[n, r] = sum_{cells c in row r of grid n} sum_k k P[c, k]

Library primitives used as steps: numpy.exp and numpy.bincount (a weighted
histogram, i.e. the per-group sum).
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    pos = z >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-z[pos]))
    e = np.exp(z[~pos])
    out[~pos] = e / (1.0 + e)
    return out


def soft_mask(x, gid, theta, tau):
    x = np.asarray(x, np.float64)
    th = np.asarray(theta, np.float64)[np.asarray(gid)]
    return sigmoid((x - th) / float(tau))


def dmask_dz(x, gid, theta, tau):
    """m (1 - m), computed as e / (1 + e)^2 with e = exp(-|z|) (no cancellation)."""
    x = np.asarray(x, np.float64)
    th = np.asarray(theta, np.float64)[np.asarray(gid)]
    z = (x - th) / float(tau)
    e = np.exp(-np.abs(z))
    return e / (1.0 + e) ** 2


def soft_filter_fwd(x, gid, theta, tau):
    return soft_mask(x, gid, theta, tau)


def soft_filter_bwd(x, gid, theta, tau, n_groups, grad_m):
    s = dmask_dz(x, gid, theta, tau)
    w = np.asarray(grad_m, np.float64) * s
    dtheta = -np.bincount(gid, weights=w, minlength=n_groups) / float(tau)
    dx = w / float(tau)
    return dtheta, dx


def soft_agg_fwd(x, v, gid, theta, tau, n_groups):
    m = soft_mask(x, gid, theta, tau)
    S = np.bincount(gid, weights=np.asarray(v, np.float64) * m, minlength=n_groups)
    Cn = np.bincount(gid, weights=m, minlength=n_groups)
    return S, Cn


def soft_agg_bwd(x, v, gid, theta, tau, n_groups, gS, gC):
    """Returns (dtheta [G], dv [n], dx [n]) for upstream gradients gS, gC."""
    gS = np.asarray(gS, np.float64)
    gC = np.asarray(gC, np.float64)
    v = np.asarray(v, np.float64)
    m = soft_mask(x, gid, theta, tau)
    s = dmask_dz(x, gid, theta, tau)
    dL_dm = gS[gid] * v + gC[gid]
    w = dL_dm * s
    dtheta = -np.bincount(gid, weights=w, minlength=n_groups) / float(tau)
    dx = w / float(tau)
    dv = gS[gid] * m
    return dtheta, dv, dx


def hard_agg(x, v, gid, theta, n_groups):
    """The exact query the soft one relaxes: rows with x > theta[g]."""
    keep = np.asarray(x, np.float64) > np.asarray(theta, np.float64)[gid]
    S = np.bincount(gid, weights=np.where(keep, np.asarray(v, np.float64), 0.0), minlength=n_groups)
    Cn = np.bincount(gid, weights=keep.astype(np.float64), minlength=n_groups)
    return S, Cn


# ---------------------------------------------------------------- PE group-by

def pe_groupby_fwd(P, grid_h: int = 4, grid_w: int = 4):
    """P: [n_cells, K] probabilities, cells of grid n are rows
    n*grid_h*grid_w .. in row-major (row, column) order.
    Returns cnt [n_grids, K], rsum [n_grids, grid_h]."""
    P = np.asarray(P, np.float64)
    K = P.shape[1]
    Pg = P.reshape(-1, grid_h, grid_w, K)
    cnt = Pg.sum(axis=(1, 2))
    rsum = (Pg * np.arange(K, dtype=np.float64)).sum(axis=(2, 3))
    return cnt, rsum


def pe_groupby_bwd(dcnt, drsum, grid_h: int = 4, grid_w: int = 4):
    dcnt = np.asarray(dcnt, np.float64)
    drsum = np.asarray(drsum, np.float64)
    K = dcnt.shape[1]
    dP = dcnt[:, None, None, :] + drsum[:, :, None, None] * np.arange(K, dtype=np.float64)
    dP = np.broadcast_to(dP, (dcnt.shape[0], grid_h, grid_w, K))
    return dP.reshape(-1, K).copy()


def exact_groupby(labels, K: int = 10):
    """Exact COUNT per class and per-row SUM of class values from integer
    labels [n_grids, grid_h, grid_w] (the inference-time query, Sec. 4)."""
    labels = np.asarray(labels)
    n = labels.shape[0]
    cnt = np.zeros((n, K), np.int64)
    for k in range(K):
        cnt[:, k] = (labels == k).sum(axis=(1, 2))
    rsum = labels.sum(axis=2).astype(np.int64)
    return cnt, rsum


# ------------------------------------------------- two-attribute PE group-by

def pe_groupby2_fwd(Pa, Pb, cells: int = 16):
    """GROUP BY (a, b) COUNT over two probability-encoded attributes of the
    same cells (the paper's Digit x Size grouping): per grid,
    cnt[a, b] = sum over the grid's cells c of Pa[c, a] * Pb[c, b].
    Pa [n_cells, Ka], Pb [n_cells, Kb] -> cnt [n_grids, Ka, Kb]."""
    Pa = np.asarray(Pa, np.float64)
    Pb = np.asarray(Pb, np.float64)
    n = Pa.shape[0] // cells
    Pa = Pa.reshape(n, cells, -1)
    Pb = Pb.reshape(n, cells, -1)
    cnt = np.zeros((n, Pa.shape[2], Pb.shape[2]))
    for c in range(cells):
        cnt += Pa[:, c, :, None] * Pb[:, c, None, :]
    return cnt


def pe_groupby2_bwd(dcnt, Pa, Pb, cells: int = 16):
    """Adjoint of pe_groupby2_fwd: dPa[c, a] = sum_b dcnt[a, b] Pb[c, b],
    dPb[c, b] = sum_a dcnt[a, b] Pa[c, a] (c in the grid of dcnt)."""
    dcnt = np.asarray(dcnt, np.float64)
    Pa = np.asarray(Pa, np.float64)
    Pb = np.asarray(Pb, np.float64)
    n = dcnt.shape[0]
    Pa3 = Pa.reshape(n, cells, -1)
    Pb3 = Pb.reshape(n, cells, -1)
    dPa = np.zeros_like(Pa3)
    dPb = np.zeros_like(Pb3)
    for c in range(cells):
        dPa[:, c, :] = (dcnt * Pb3[:, c, None, :]).sum(axis=2)
        dPb[:, c, :] = (dcnt * Pa3[:, c, :, None]).sum(axis=1)
    return dPa.reshape(Pa.shape), dPb.reshape(Pb.shape)


def exact_groupby2(a_labels, b_labels, Ka: int = 10, Kb: int = 2):
    """Exact COUNT per (a, b) pair per grid from integer labels
    [n_grids, grid_h, grid_w] of both attributes: [n_grids, Ka, Kb]."""
    a = np.asarray(a_labels).reshape(len(a_labels), -1)
    b = np.asarray(b_labels).reshape(len(b_labels), -1)
    cnt = np.zeros((a.shape[0], Ka, Kb), np.int64)
    for i in range(Ka):
        for j in range(Kb):
            cnt[:, i, j] = ((a == i) & (b == j)).sum(axis=1)
    return cnt
