"""Learning from label proportions (Sec. 5.3) and its label-DP variant
(Sec. 5.4) on the GPU.

A linear table-valued function classifies every row; the per-bag
GROUP BY class COUNT runs softly (softmax in place of argmax), and the MSE
between the soft counts and the bags' count labels is minimised with Adam.
The count labels are the exact per-bag counts, optionally passed through the
Laplace mechanism.  Every step runs in libtdp.so (tdp_llp.h); torch provides
device buffers and the stream only.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .ops import _ptr, _require_cuda, _stream

DP_SENSITIVITY = 2.0  # L1 change of a bag's count vector when one row's label changes


def n_bags(n: int, B: int) -> int:
    return (n + B - 1) // B


def counts(labels: torch.Tensor, B: int, K: int = 2, noise: torch.Tensor | None = None,
           eps: float | None = None, status: torch.Tensor | None = None) -> torch.Tensor:
    """Count labels of the bags: exact per-bag class counts, plus the Laplace
    mechanism (scale 2 / eps times the standard Laplace draws `noise`) when
    noise is given."""
    _require_cuda(labels, noise)
    n = labels.shape[0]
    out = torch.empty((n_bags(n, B), K), dtype=torch.float32, device=labels.device)
    scale = DP_SENSITIVITY / eps if noise is not None else 0.0
    L.call("tdp_llp_counts", _ptr(labels), n, K, B, _ptr(noise), float(scale), _ptr(out), _ptr(status), _stream())
    return out


def predict(X: torch.Tensor, W: torch.Tensor, b: torch.Tensor, ref: torch.Tensor | None = None):
    """Hard classifier (first arg-max of the logits): (labels, n_errors or
    None) with n_errors a device int64 scalar when ref labels are given."""
    _require_cuda(X, W, b, ref)
    n, d = X.shape
    K = W.shape[0]
    lab = torch.empty(n, dtype=torch.int32, device=X.device)
    err = torch.zeros(1, dtype=torch.int64, device=X.device) if ref is not None else None
    L.call("tdp_llp_predict", _ptr(X), n, d, K, _ptr(W), _ptr(b), _ptr(lab), _ptr(ref), _ptr(err), _stream())
    return lab, err


class LLPTrainer:
    """Full-batch training of the linear classifier from bag counts:
    each step is one fused forward + backward pass over all rows
    (tdp_llp_step) and one Adam update of W and b (tdp_adam_step)."""

    def __init__(self, X: torch.Tensor, targets: torch.Tensor, B: int, W0, b0, lr: float = 0.05,
                 betas=(0.9, 0.999), eps: float = 1e-8):
        _require_cuda(X, targets)
        self.X, self.targets, self.B = X.contiguous(), targets.contiguous(), int(B)
        self.n, self.d = X.shape
        dev = X.device
        self.W = torch.as_tensor(np.asarray(W0, np.float32)).to(dev).contiguous()
        self.b = torch.as_tensor(np.asarray(b0, np.float32)).to(dev).contiguous()
        self.K = self.W.shape[0]
        if targets.shape != (n_bags(self.n, self.B), self.K):
            raise ValueError("targets must be [n_bags, K]")
        self.dW, self.db = torch.zeros_like(self.W), torch.zeros_like(self.b)
        self.mW, self.vW = torch.zeros_like(self.W), torch.zeros_like(self.W)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        # device status word (bounded waits of the bulk-copy pipeline)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.cnt = torch.empty_like(self.targets)
        wsb = L.lib().tdp_llp_step_workspace(self.n, self.d, self.K, self.B)
        self.ws = torch.empty(max(16, int(wsb)), dtype=torch.uint8, device=dev)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.t = 0
        self._arr = lambda ts: (C.c_void_p * 2)(*[t.data_ptr() for t in ts])  # noqa: E731

    def forward_backward(self, cnt_out: bool = False) -> torch.Tensor:
        L.call("tdp_llp_step", _ptr(self.X), self.n, self.d, self.K, self.B, _ptr(self.W), _ptr(self.b),
               _ptr(self.targets), _ptr(self.cnt) if cnt_out else None, _ptr(self.loss), _ptr(self.dW),
               _ptr(self.db), _ptr(self.ws), self.ws.numel(), _ptr(self.status), _stream())
        return self.loss

    def adam(self) -> None:
        self.t += 1
        sizes = (C.c_int64 * 2)(self.W.numel(), self.b.numel())
        L.call("tdp_adam_step", self._arr([self.W, self.b]), self._arr([self.dW, self.db]),
               self._arr([self.mW, self.mb]), self._arr([self.vW, self.vb]), None, sizes, 2, self.t,
               float(self.lr), float(self.betas[0]), float(self.betas[1]), float(self.eps), _stream())

    def step(self) -> torch.Tensor:
        loss = self.forward_backward()
        self.adam()
        return loss
