"""torch.autograd.Function wrappers of the soft operators (Sec. 4).

Forward and backward both run the library's kernels; only the inputs are
saved (the mask is recomputed in the backward kernel, never stored).
"""
from __future__ import annotations

import torch

from . import ops


class SoftAgg(torch.autograd.Function):
    """(S, C) = soft_groupby(x, v, gid; theta, tau):
    S[g] = sum v_i m_i, C[g] = sum m_i, m_i = sigmoid((x_i - theta[g_i]) / tau)."""

    @staticmethod
    def forward(ctx, x, v, gid, theta, tau: float):
        S, C = ops.soft_agg_fwd(x, v, gid, theta, tau)
        ctx.save_for_backward(x, v, gid, theta)
        ctx.tau = tau
        return S, C

    @staticmethod
    def backward(ctx, gS, gC):
        x, v, gid, theta = ctx.saved_tensors
        gS = torch.zeros_like(theta) if gS is None else gS.contiguous()
        gC = torch.zeros_like(theta) if gC is None else gC.contiguous()
        gth, gv, gx = ops.soft_agg_bwd(x, v, gid, theta, ctx.tau, gS, gC,
                                       need_v=ctx.needs_input_grad[1], need_x=ctx.needs_input_grad[0])
        return gx, gv, None, gth, None


class SoftFilter(torch.autograd.Function):
    """m = sigmoid((x - theta[gid]) / tau) (the relaxed WHERE x > theta)."""

    @staticmethod
    def forward(ctx, x, gid, theta, tau: float):
        m = ops.soft_filter_fwd(x, gid, theta, tau)
        ctx.save_for_backward(x, gid, theta)
        ctx.tau = tau
        return m

    @staticmethod
    def backward(ctx, gm):
        x, gid, theta = ctx.saved_tensors
        gth, gx = ops.soft_filter_bwd(x, gid, theta, ctx.tau, gm.contiguous(), need_x=ctx.needs_input_grad[0])
        return gx, None, gth, None
