"""The trainable glyph query (Sec. 3 training loop, Sec. 4, Sec. 5.5).

A grid image of 4x4 glyph cells goes through the CNN (the table-valued
function of the paper's MNISTGrid example), the per-cell class probabilities
(the PE column) feed the soft group-by (per-class COUNT and per-row SUM of
class values), and the MSE against the exact query on true labels is
minimised with Adam, end to end, by the library's kernels.  At inference the
exact query (argmax, integer COUNT/SUM) replaces the soft one.

Only device buffers and the stream come from torch; every layer, loss,
gradient and optimiser update runs in libtdp.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .ops import _ptr, _stream

PARAMS = ("conv1_w", "conv1_b", "conv2_w", "conv2_b", "fc1_w", "fc1_b", "fc2_w", "fc2_b")
BF16_COPIES = ("conv2_w", "fc1_w")  # operands of the tensor-core layers
CELLS = 16
NPRED = 14


class GlyphQuery:
    def __init__(self, params: dict, device="cuda", lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8,
                 warmup: int = 400):
        """Adam with a linear learning-rate warmup over `warmup` steps.  The
        paper's loop uses Adam at lr 0.01; on this network that diverges, and
        lr 1e-3 without warmup lets the softmax of class 0 (value 0, invisible
        to the row sums) saturate and collapse into class 1."""
        self.dev = torch.device(device)
        self.p = {k: torch.as_tensor(np.asarray(params[k], np.float32)).to(self.dev).contiguous() for k in PARAMS}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.bf = {k: torch.empty(self.p[k].shape, dtype=torch.bfloat16, device=self.dev) for k in BF16_COPIES}
        for k in BF16_COPIES:
            L.call("tdp_f32_to_bf16", _ptr(self.p[k]), self.p[k].numel(), _ptr(self.bf[k]), _stream())
        self.lr, self.betas, self.eps, self.warmup = lr, betas, eps, warmup
        self.t = 0
        self._buf = {}
        # device status word of the kernels that wait on the device (bounded waits)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)

    # -------------------------------------------------------------- buffers
    def _buffers(self, n_grids: int) -> dict:
        b = self._buf.get(n_grids)
        if b is not None:
            return b
        nc = n_grids * CELLS
        d = self.dev
        lib = L.lib()
        ws = max(lib.tdp_cnn_fc1_fwd_workspace(nc), lib.tdp_cnn_head_workspace(n_grids),
                 lib.tdp_cnn_fc1_bwd_workspace(nc), lib.tdp_cnn_conv2_bwd_workspace(nc),
                 lib.tdp_cnn_conv1_bwd_workspace(nc))
        b = {
            "y1": torch.empty((nc, 26, 26, 32), dtype=torch.bfloat16, device=d),
            "y2": torch.empty((nc, 9216), dtype=torch.bfloat16, device=d),
            "argmax": torch.empty((nc, 9216), dtype=torch.uint8, device=d),
            "h1": torch.empty((nc, 128), dtype=torch.bfloat16, device=d),
            "dh1": torch.empty((nc, 128), dtype=torch.bfloat16, device=d),
            "dy2p": torch.empty((nc, 9216), dtype=torch.bfloat16, device=d),
            "dz1": torch.empty((nc, 26, 26, 32), dtype=torch.bfloat16, device=d),
            "logits": torch.empty((nc, 10), dtype=torch.float32, device=d),
            "P": torch.empty((nc, 10), dtype=torch.float32, device=d),
            "pred": torch.empty((n_grids, NPRED), dtype=torch.float32, device=d),
            "loss": torch.empty(1, dtype=torch.float32, device=d),
            "labels": torch.empty(nc, dtype=torch.int32, device=d),
            "cnt": torch.empty((n_grids, 10), dtype=torch.int64, device=d),
            "rsum": torch.empty((n_grids, 4), dtype=torch.int64, device=d),
            "ws": torch.empty(int(ws), dtype=torch.uint8, device=d),
        }
        self._buf[n_grids] = b
        return b

    # -------------------------------------------------------------- forward
    def forward(self, grids: torch.Tensor, targets: torch.Tensor | None = None,
                loss_out: torch.Tensor | None = None) -> dict:
        """Forward (and, with targets, the loss backward down to dh1).  The
        mean loss goes to b["loss"], or to the one-element fp32 device tensor
        loss_out when given."""
        n = grids.shape[0]
        nc = n * CELLS
        b = self._buffers(n)
        s = _stream()
        p = self.p
        ws, wsn = _ptr(b["ws"]), b["ws"].numel()
        L.call("tdp_cnn_conv1_fwd", _ptr(grids), n, _ptr(p["conv1_w"]), _ptr(p["conv1_b"]), _ptr(b["y1"]), s)
        L.call("tdp_cnn_conv2_pool_fwd", _ptr(b["y1"]), nc, _ptr(self.bf["conv2_w"]), _ptr(p["conv2_b"]),
               _ptr(b["y2"]), _ptr(b["argmax"]), _ptr(self.status), s)
        L.call("tdp_cnn_fc1_fwd", _ptr(b["y2"]), nc, _ptr(self.bf["fc1_w"]), _ptr(p["fc1_b"]), _ptr(b["h1"]), ws,
               wsn, _ptr(self.status), s)
        g = self.g
        L.call("tdp_cnn_head", _ptr(b["h1"]), n, _ptr(p["fc2_w"]), _ptr(p["fc2_b"]), _ptr(targets),
               _ptr(b["logits"]), _ptr(b["P"]), _ptr(b["pred"]),
               _ptr(b["dh1"]) if targets is not None else None,
               _ptr(g["fc2_w"]) if targets is not None else None,
               _ptr(g["fc2_b"]) if targets is not None else None,
               _ptr(loss_out if loss_out is not None else b["loss"]) if targets is not None else None, ws, wsn,
               s)
        return b

    def backward(self, grids: torch.Tensor) -> None:
        """Parameter gradients into self.g (after forward with targets)."""
        n = grids.shape[0]
        nc = n * CELLS
        b = self._buffers(n)
        s = _stream()
        g = self.g
        ws, wsn = _ptr(b["ws"]), b["ws"].numel()
        L.call("tdp_cnn_fc1_bwd", _ptr(b["dh1"]), _ptr(b["y2"]), _ptr(self.bf["fc1_w"]), nc, _ptr(b["dy2p"]),
               _ptr(g["fc1_w"]), _ptr(g["fc1_b"]), ws, wsn, _ptr(self.status), s)
        L.call("tdp_cnn_conv2_bwd", _ptr(b["dy2p"]), _ptr(b["argmax"]), _ptr(b["y1"]), _ptr(self.bf["conv2_w"]), nc,
               _ptr(b["dz1"]), _ptr(g["conv2_w"]), _ptr(g["conv2_b"]), ws, wsn, _ptr(self.status), s)
        L.call("tdp_cnn_conv1_bwd", _ptr(b["dz1"]), _ptr(grids), nc, _ptr(g["conv1_w"]), _ptr(g["conv1_b"]), ws,
               wsn, s)

    def adam(self) -> None:
        self.t += 1
        k = list(self.p)
        n = len(k)
        arr = lambda ts: (C.c_void_p * n)(*[t.data_ptr() for t in ts])  # noqa: E731
        copies = (C.c_void_p * n)(*[self.bf[x].data_ptr() if x in self.bf else 0 for x in k])
        sizes = (C.c_int64 * n)(*[self.p[x].numel() for x in k])
        lr = self.lr * min(1.0, self.t / self.warmup) if self.warmup else self.lr
        L.call("tdp_adam_step", arr([self.p[x] for x in k]), arr([self.g[x] for x in k]),
               arr([self.m[x] for x in k]), arr([self.v[x] for x in k]), copies, sizes, len(k), self.t,
               float(lr), float(self.betas[0]), float(self.betas[1]), float(self.eps), _stream())

    def train_step(self, grids: torch.Tensor, targets: torch.Tensor,
                   loss_out: torch.Tensor | None = None) -> torch.Tensor:
        """One step of the paper's training loop: query forward, MSE loss,
        backward through the soft query into the CNN, Adam.  Returns the
        device loss (mean squared error): loss_out when given (a one-element
        fp32 device tensor, e.g. a slot of a loss history), else the query's
        own loss buffer, which the next step overwrites."""
        b = self.forward(grids, targets, loss_out)
        self.backward(grids)
        self.adam()
        return loss_out if loss_out is not None else b["loss"]

    # -------------------------------------------------------------- inference
    def soft_query(self, grids: torch.Tensor) -> torch.Tensor:
        return self.forward(grids)["pred"]

    def exact_query(self, grids: torch.Tensor):
        """Exact query on argmax labels: (labels [n*16], cnt [n,10], rsum [n,4])."""
        b = self.forward(grids)
        n = grids.shape[0]
        L.call("tdp_exact_pe_count", _ptr(b["logits"]), n, 10, 4, 4, _ptr(b["labels"]), _ptr(b["cnt"]),
               _ptr(b["rsum"]), _stream())
        return b["labels"], b["cnt"], b["rsum"]

    def state(self) -> dict:
        """Checkpoint: parameters, Adam moments and step (host copies)."""
        out = {"t": self.t}
        for k in self.p:
            out["p." + k] = self.p[k].cpu()
            out["m." + k] = self.m[k].cpu()
            out["v." + k] = self.v[k].cpu()
        return out

    def load_state(self, st: dict) -> None:
        self.t = int(st["t"])
        for k in self.p:
            self.p[k].copy_(st["p." + k])
            self.m[k].copy_(st["m." + k])
            self.v[k].copy_(st["v." + k])
        for k in BF16_COPIES:
            L.call("tdp_f32_to_bf16", _ptr(self.p[k]), self.p[k].numel(), _ptr(self.bf[k]), _stream())


SIZE_PARAMS = ("fc2s_w", "fc2s_b")
NPRED2 = 20


class GlyphQuery2(GlyphQuery):
    """The Digit x Size query: the same CNN trunk with a second head (fc2s,
    128 -> 2 size classes) on the hidden layer; the soft COUNT of every
    (digit, size) pair per grid (20 outputs) is trained with an MSE against
    the exact pair counts on true labels, end to end through both heads."""

    def __init__(self, params: dict, size_params: dict, device="cuda", **kw):
        super().__init__(params, device, **kw)
        for k in SIZE_PARAMS:
            self.p[k] = torch.as_tensor(np.asarray(size_params[k], np.float32)).to(self.dev).contiguous()
            self.m[k] = torch.zeros_like(self.p[k])
            self.v[k] = torch.zeros_like(self.p[k])
            self.g[k] = torch.zeros_like(self.p[k])

    def _buffers(self, n_grids: int) -> dict:
        b = self._buf.get(n_grids)
        if b is not None and "pred2" in b:
            return b
        b = super()._buffers(n_grids)
        nc = n_grids * CELLS
        d = self.dev
        hw = L.lib().tdp_cnn_head2_workspace(n_grids)
        if b["ws"].numel() < hw:
            b["ws"] = torch.empty(int(hw), dtype=torch.uint8, device=d)
        b.update({
            "logits_s": torch.empty((nc, 2), dtype=torch.float32, device=d),
            "Ps": torch.empty((nc, 2), dtype=torch.float32, device=d),
            "pred2": torch.empty((n_grids, NPRED2), dtype=torch.float32, device=d),
            "labels_s": torch.empty(nc, dtype=torch.int32, device=d),
            "cnt2": torch.empty((n_grids, 10, 2), dtype=torch.int64, device=d),
        })
        return b

    def forward(self, grids: torch.Tensor, targets: torch.Tensor | None = None,
                loss_out: torch.Tensor | None = None) -> dict:
        n = grids.shape[0]
        nc = n * CELLS
        b = self._buffers(n)
        s = _stream()
        p = self.p
        ws, wsn = _ptr(b["ws"]), b["ws"].numel()
        L.call("tdp_cnn_conv1_fwd", _ptr(grids), n, _ptr(p["conv1_w"]), _ptr(p["conv1_b"]), _ptr(b["y1"]), s)
        L.call("tdp_cnn_conv2_pool_fwd", _ptr(b["y1"]), nc, _ptr(self.bf["conv2_w"]), _ptr(p["conv2_b"]),
               _ptr(b["y2"]), _ptr(b["argmax"]), _ptr(self.status), s)
        L.call("tdp_cnn_fc1_fwd", _ptr(b["y2"]), nc, _ptr(self.bf["fc1_w"]), _ptr(p["fc1_b"]), _ptr(b["h1"]), ws,
               wsn, _ptr(self.status), s)
        g = self.g
        tr = targets is not None
        L.call("tdp_cnn_head2", _ptr(b["h1"]), n, _ptr(p["fc2_w"]), _ptr(p["fc2_b"]), _ptr(p["fc2s_w"]),
               _ptr(p["fc2s_b"]), _ptr(targets), _ptr(b["logits"]), _ptr(b["logits_s"]), _ptr(b["P"]),
               _ptr(b["Ps"]), _ptr(b["pred2"]), _ptr(b["dh1"]) if tr else None,
               _ptr(g["fc2_w"]) if tr else None, _ptr(g["fc2_b"]) if tr else None,
               _ptr(g["fc2s_w"]) if tr else None, _ptr(g["fc2s_b"]) if tr else None,
               _ptr(loss_out if loss_out is not None else b["loss"]) if tr else None, ws, wsn, s)
        return b

    def soft_query(self, grids: torch.Tensor) -> torch.Tensor:
        return self.forward(grids)["pred2"]

    def exact_query(self, grids: torch.Tensor):
        """Exact pair query on argmax labels: (digits [n*16], sizes [n*16],
        cnt [n, 10, 2])."""
        b = self.forward(grids)
        n = grids.shape[0]
        L.call("tdp_exact_pe_count2", _ptr(b["logits"]), 10, _ptr(b["logits_s"]), 2, n, CELLS, _ptr(b["labels"]),
               _ptr(b["labels_s"]), _ptr(b["cnt2"]), _stream())
        return b["labels"], b["labels_s"], b["cnt2"]


def pe_groupby2_fwd(Pa: torch.Tensor, Pb: torch.Tensor, n_grids: int, cells: int = CELLS):
    Ka, Kb = Pa.shape[1], Pb.shape[1]
    cnt = torch.empty((n_grids, Ka, Kb), dtype=torch.float32, device=Pa.device)
    L.call("tdp_pe_groupby2_fwd", _ptr(Pa), Ka, _ptr(Pb), Kb, n_grids, cells, _ptr(cnt), _stream())
    return cnt


def pe_groupby2_bwd(dcnt: torch.Tensor, Pa: torch.Tensor, Pb: torch.Tensor, cells: int = CELLS):
    n, Ka, Kb = dcnt.shape
    dPa = torch.empty_like(Pa)
    dPb = torch.empty_like(Pb)
    L.call("tdp_pe_groupby2_bwd", _ptr(dcnt), _ptr(Pa), Ka, _ptr(Pb), Kb, n, cells, _ptr(dPa), _ptr(dPb),
           _stream())
    return dPa, dPb


def exact_count2(logits_a: torch.Tensor, logits_b: torch.Tensor, n_grids: int, cells: int = CELLS):
    Ka, Kb = logits_a.shape[1], logits_b.shape[1]
    la = torch.empty(n_grids * cells, dtype=torch.int32, device=logits_a.device)
    lb = torch.empty(n_grids * cells, dtype=torch.int32, device=logits_a.device)
    cnt = torch.empty((n_grids, Ka, Kb), dtype=torch.int64, device=logits_a.device)
    L.call("tdp_exact_pe_count2", _ptr(logits_a), Ka, _ptr(logits_b), Kb, n_grids, cells, _ptr(la), _ptr(lb),
           _ptr(cnt), _stream())
    return la, lb, cnt


def pe_groupby_fwd(P: torch.Tensor, n_grids: int, K: int = 10, gh: int = 4, gw: int = 4):
    cnt = torch.empty((n_grids, K), dtype=torch.float32, device=P.device)
    rsum = torch.empty((n_grids, gh), dtype=torch.float32, device=P.device)
    L.call("tdp_pe_groupby_fwd", _ptr(P), n_grids, K, gh, gw, _ptr(cnt), _ptr(rsum), _stream())
    return cnt, rsum


def pe_groupby_bwd(dcnt: torch.Tensor, drsum: torch.Tensor, K: int = 10, gh: int = 4, gw: int = 4):
    n = dcnt.shape[0]
    dP = torch.empty((n * gh * gw, K), dtype=torch.float32, device=dcnt.device)
    L.call("tdp_pe_groupby_bwd", _ptr(dcnt), _ptr(drsum), n, K, gh, gw, _ptr(dP), _stream())
    return dP


def exact_count(logits: torch.Tensor, n_grids: int, K: int = 10, gh: int = 4, gw: int = 4):
    labels = torch.empty(n_grids * gh * gw, dtype=torch.int32, device=logits.device)
    cnt = torch.empty((n_grids, K), dtype=torch.int64, device=logits.device)
    rsum = torch.empty((n_grids, gh), dtype=torch.int64, device=logits.device)
    L.call("tdp_exact_pe_count", _ptr(logits), n_grids, K, gh, gw, _ptr(labels), _ptr(cnt), _ptr(rsum), _stream())
    return labels, cnt, rsum
