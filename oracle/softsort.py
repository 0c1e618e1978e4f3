"""fp64 oracle for a soft ORDER BY ... LIMIT k (a relaxed sort and top-k).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4 makes discrete operators trainable by relaxing them: a logistic
function stands in for the step function of a comparison.  The paper names
sorting and top-k among the operators one may relax this way but gives no
formula; the reading taken here relaxes every comparison of a rank with the
same logistic function as the soft filter:

  rank (descending, 1-based) of row i in its group g:
      r_i  = 1 + sum_{j in g, j != i} sigma((x_j - x_i) / tau)
  top-k membership:  m_i = sigma((k + 1/2 - r_i) / tau_r)
  soft top-k sum of a payload v per group:  S_g = sum_{i in g} m_i v_i

As tau -> 0 the rank counts the rows with larger x (a tie counts 1/2), and
as tau_r -> 0 the membership becomes the indicator rank <= k, so S_g becomes
the SUM over the group's top k rows.  The exact operator at inference ranks
ties by position (the earlier row first) and keeps the rows of rank <= k.

Adjoints (s_ij = sigma'((x_j - x_i) / tau) / tau, symmetric in i and j):
  dm_i = dS_g v_i (+ a given dm_i),  dv_i = dS_g m_i
  dr_i = -dm_i m_i (1 - m_i) / tau_r (+ a given dr_i)
  dx_i = sum_{j != i} s_ij (dr_j - dr_i)

Groups are runs of consecutive rows: rows offsets[g] .. offsets[g+1] - 1.
Library primitives used as steps: numpy.exp (through soft.sigmoid), sums.
"""
from __future__ import annotations

import numpy as np

from .soft import sigmoid


def _groups(offsets):
    o = np.asarray(offsets, np.int64)
    return [(int(o[g]), int(o[g + 1])) for g in range(len(o) - 1)]


def soft_rank(x, offsets, tau: float):
    x = np.asarray(x, np.float64)
    r = np.empty_like(x)
    for a, b in _groups(offsets):
        xs = x[a:b]
        z = (xs[None, :] - xs[:, None]) / tau  # z[i, j] = (x_j - x_i) / tau
        s = sigmoid(z)
        np.fill_diagonal(s, 0.0)
        r[a:b] = 1.0 + s.sum(axis=1)
    return r


def soft_topk_fwd(x, v, offsets, k: int, tau: float, tau_r: float):
    """(r, m, S): soft ranks, soft top-k membership, soft top-k sum per group."""
    r = soft_rank(x, offsets, tau)
    m = sigmoid((k + 0.5 - r) / tau_r)
    v = np.asarray(v, np.float64)
    S = np.array([np.sum(m[a:b] * v[a:b]) for a, b in _groups(offsets)])
    return r, m, S


def soft_topk_bwd(x, v, offsets, k: int, tau: float, tau_r: float, m, dS=None, dm=None, dr=None):
    """(dx, dv) of the soft top-k given upstream dS [G], dm [n], dr [n]
    (each optional)."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    m = np.asarray(m, np.float64)
    n = x.shape[0]
    dmv = np.zeros(n) if dm is None else np.asarray(dm, np.float64).copy()
    dv = np.zeros(n)
    if dS is not None:
        for g, (a, b) in enumerate(_groups(offsets)):
            dmv[a:b] += dS[g] * v[a:b]
            dv[a:b] = dS[g] * m[a:b]
    drv = -dmv * m * (1.0 - m) / tau_r
    if dr is not None:
        drv = drv + np.asarray(dr, np.float64)
    dx = np.zeros(n)
    for a, b in _groups(offsets):
        xs = x[a:b]
        sg = sigmoid((xs[None, :] - xs[:, None]) / tau)
        s = sg * (1.0 - sg) / tau
        np.fill_diagonal(s, 0.0)
        d = drv[a:b]
        dx[a:b] = s @ d - d * s.sum(axis=1)
    return dx, dv


def exact_rank(x, offsets):
    """1 + #{j in g : x_j > x_i, or x_j == x_i and j < i} (ties by position)."""
    x = np.asarray(x)
    r = np.empty(x.shape[0], np.int64)
    for a, b in _groups(offsets):
        xs = x[a:b]
        idx = np.arange(b - a)
        gt = xs[None, :] > xs[:, None]
        tie = (xs[None, :] == xs[:, None]) & (idx[None, :] < idx[:, None])
        r[a:b] = 1 + (gt | tie).sum(axis=1)
    return r


def exact_topk_sum(x, v, offsets, k: int):
    r = exact_rank(x, offsets)
    v = np.asarray(v, np.float64)
    return np.array([np.sum(v[a:b][r[a:b] <= k]) for a, b in _groups(offsets)])
