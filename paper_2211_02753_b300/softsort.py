"""Soft ORDER BY ... LIMIT k per group (Sec. 4's logistic relaxation of
comparisons applied to ranks) and the exact operator, on the GPU.

  r_i = 1 + sum_{j in g, j != i} sigmoid((x_j - x_i) / tau)   (descending rank)
  m_i = sigmoid((k + 1/2 - r_i) / tau_r)                       (top-k membership)
  S_g = sum_{i in g} m_i v_i                                   (soft top-k SUM)

Groups are runs of consecutive rows given by int64 offsets [G + 1].  Every
step runs in libtdp.so (include/tdp_softsort.h).
"""
from __future__ import annotations

import torch

from . import _lib as L
from .ops import _ptr, _require_cuda, _stream


def _max_group(offsets: torch.Tensor, max_group: int | None) -> int:
    if max_group is not None:
        return int(max_group)
    return max(1, int((offsets[1:] - offsets[:-1]).max().item())) if offsets.numel() > 1 else 1


def soft_topk_fwd(x, v, offsets, k: int, tau: float, tau_r: float = 0.5, max_group: int | None = None,
                  status: torch.Tensor | None = None):
    """(rank, mask, sum): soft ranks and membership [n], soft top-k sums [G]
    (None without v).  max_group (the largest group's size) is read from
    offsets when not given (a device sync)."""
    _require_cuda(x, v, offsets)
    n, G = x.shape[0], offsets.shape[0] - 1
    mg = _max_group(offsets, max_group)
    rank = torch.empty(n, dtype=torch.float32, device=x.device)
    mask = torch.empty(n, dtype=torch.float32, device=x.device)
    ssum = torch.empty(G, dtype=torch.float32, device=x.device) if v is not None else None
    L.call("tdp_soft_topk_fwd", _ptr(x), _ptr(v), n, _ptr(offsets), G, mg, int(k), float(tau), float(tau_r),
           _ptr(rank), _ptr(mask), _ptr(ssum), _ptr(status), _stream())
    return rank, mask, ssum


def soft_topk_bwd(x, v, offsets, k: int, tau: float, tau_r: float, mask, dsum=None, dmask=None, drank=None,
                  max_group: int | None = None, status: torch.Tensor | None = None):
    """(dx, dv): gradients of the soft top-k given upstream dsum [G],
    dmask [n], drank [n] (each optional; dv only with dsum and v)."""
    _require_cuda(x, v, offsets, mask, dsum, dmask, drank)
    n, G = x.shape[0], offsets.shape[0] - 1
    mg = _max_group(offsets, max_group)
    dx = torch.empty(n, dtype=torch.float32, device=x.device)
    dv = torch.empty(n, dtype=torch.float32, device=x.device) if (dsum is not None and v is not None) else None
    ws = torch.empty(int(L.lib().tdp_soft_topk_workspace(n)), dtype=torch.uint8, device=x.device)
    L.call("tdp_soft_topk_bwd", _ptr(x), _ptr(v), n, _ptr(offsets), G, mg, int(k), float(tau), float(tau_r),
           _ptr(mask), _ptr(dsum), _ptr(dmask), _ptr(drank), _ptr(dx), _ptr(dv), _ptr(ws), ws.numel(),
           _ptr(status), _stream())
    return dx, dv


def exact_topk(x, v, offsets, k: int, max_group: int | None = None, status: torch.Tensor | None = None):
    """(rank int32 [n], sum float64 [G] or None): exact descending ranks with
    ties by position and the SUM of v over each group's rows of rank <= k."""
    _require_cuda(x, v, offsets)
    n, G = x.shape[0], offsets.shape[0] - 1
    mg = _max_group(offsets, max_group)
    rank = torch.empty(n, dtype=torch.int32, device=x.device)
    ssum = torch.empty(G, dtype=torch.float64, device=x.device) if v is not None else None
    L.call("tdp_exact_topk", _ptr(x), _ptr(v), n, _ptr(offsets), G, mg, int(k), _ptr(rank), _ptr(ssum),
           _ptr(status), _stream())
    return rank, ssum


class SoftTopKSum(torch.autograd.Function):
    """S = soft top-k SUM of v by x descending, per group; differentiable in
    x and v."""

    @staticmethod
    def forward(ctx, x, v, offsets, k: int, tau: float, tau_r: float, max_group: int):
        _, mask, S = soft_topk_fwd(x, v, offsets, k, tau, tau_r, max_group)
        ctx.save_for_backward(x, v, offsets, mask)
        ctx.args = (k, tau, tau_r, max_group)
        return S

    @staticmethod
    def backward(ctx, dS):
        x, v, offsets, mask = ctx.saved_tensors
        k, tau, tau_r, mg = ctx.args
        dx, dv = soft_topk_bwd(x, v, offsets, k, tau, tau_r, mask, dsum=dS.contiguous(), max_group=mg)
        return dx, dv, None, None, None, None, None
