"""Python wrappers over the tdp C ABI (argument marshalling only).

Every function takes CUDA tensors, allocates its outputs and scratch with
torch (device memory is the only thing torch provides here), and launches the
library's kernels on the current CUDA stream.  Host-side argument errors
raise ``TdpError`` immediately; device-side errors land in a status tensor
that ``check()`` reads (this synchronises).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import TdpError

_DT = {torch.int8: L.I8, torch.uint8: L.U8, torch.int32: L.I32, torch.int64: L.I64,
       torch.float32: L.F32, torch.bfloat16: L.BF16}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tdp operators take CUDA tensors (no CPU path)")


class Col:
    """A column tensor with optional metadata bounds lo <= value <= hi."""

    def __init__(self, t: torch.Tensor, lo=None, hi=None):
        self.t = t
        self.lo = lo
        self.hi = hi


def _as_col(c):
    return c if isinstance(c, Col) else Col(c)


def col_array(cols):
    cols = [_as_col(c) for c in cols]
    _require_cuda(*[c.t for c in cols])
    arr = (L.TdpCol * max(1, len(cols)))()
    for i, c in enumerate(cols):
        t = c.t
        if not t.is_contiguous():
            raise ValueError("columns must be contiguous")
        arr[i].data = t.data_ptr()
        arr[i].dtype = _DT[t.dtype]
        arr[i].n = t.numel()
        if c.lo is not None:
            arr[i].has_bounds = 1
            arr[i].lo = int(c.lo)
            arr[i].hi = int(c.hi)
    return arr


def pred_array(preds):
    arr = (L.TdpPred * max(1, len(preds)))()
    for i, (c, op, lit) in enumerate(preds):
        arr[i].col = int(c)
        arr[i].cmp = L.CMP[op]
        arr[i].lit = int(lit)
    return arr


def agg_array(aggs):
    """aggs: list of (op, a, b, k); a/b column indices (or None)."""
    arr = (L.TdpAgg * max(1, len(aggs)))()
    for i, g in enumerate(aggs):
        op, a, b, k = (tuple(g) + (None, None, None))[:4]
        arr[i].op = L.AGG[op]
        arr[i].a = -1 if a is None else int(a)
        arr[i].b = -1 if b is None else int(b)
        arr[i].k = 0 if k is None else int(k)
    return arr


def _int_array(vals, ctype=C.c_int32):
    return (ctype * max(1, len(vals)))(*[int(v) for v in vals])


def _ptr_array(ts):
    return (C.c_void_p * max(1, len(ts)))(*[t.data_ptr() for t in ts])


class Workspace:
    """Grow-only scratch buffer reused across calls (one per device)."""

    def __init__(self):
        self._buf = {}

    def get(self, nbytes: int, device) -> torch.Tensor:
        dev = torch.device(device)
        b = self._buf.get(dev)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
            self._buf[dev] = b
        return b


_WS = Workspace()


def workspace(nbytes, device):
    return _WS.get(nbytes, device)


def new_status(device):
    return torch.zeros(1, dtype=torch.int32, device=device)


def check(status: torch.Tensor, where: str = "tdp"):
    """Reads a device status word (synchronising) and raises on an error."""
    s = int(status.item())
    if s != 0:
        raise TdpError(s, where)


def status_str(code: int) -> str:
    return L.lib().tdp_status_str(int(code)).decode()


def set_spin_limit(polls: int) -> int:
    return int(L.lib().tdp_set_spin_limit(int(polls)))


def debug_wait_flag(flag: torch.Tensor, polls: int, status: torch.Tensor):
    L.call("tdp_debug_wait_flag", _ptr(flag), int(polls), _ptr(status), _stream())


# ---------------------------------------------------------------- filter

def filter(cols, preds, n=None, capacity=None, gather=(), rowids=True, status=None, d_n=None):
    """WHERE conjunction over `cols` (list of tensors / Col).

    preds: list of (column index, op, integer literal).
    gather: column indices to gather at the qualifying rows.
    Returns dict(rowid, count, gathered, status); rowid/gathered have
    `capacity` rows, the first `count` are valid."""
    carr = col_array(cols)
    dev = _as_col(cols[0]).t.device
    n = _as_col(cols[0]).t.numel() if n is None else int(n)
    cap = n if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    rowid = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if rowids else None
    count = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    gout = [torch.empty(max(cap, 1), dtype=_as_col(cols[g]).t.dtype, device=dev) for g in gather]
    ws_n = L.lib().tdp_filter_workspace(n)
    ws = workspace(ws_n, dev)
    L.call("tdp_filter", carr, len(cols), pred_array(preds), len(preds), n, _ptr(d_n), _ptr(rowid), cap, _ptr(count),
           _int_array(gather), len(gather), _ptr_array(gout), _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"rowid": rowid, "count": count, "gathered": gout, "status": status}


# -------------------------------------------------------------- group-by

def groupby_agg(cols, key_cols, aggs, preds=(), n=None, sel=None, nsel=None, strategy="auto", capacity=None,
                status=None):
    """GROUP BY cols[key_cols] with aggregates (op, a, b, k).

    Returns dict(keys [list of tensors], aggs [list of int64 tensors],
    ngroups (device int64[1]), status)."""
    carr = col_array(cols)
    dev = _as_col(cols[0]).t.device
    if n is None:
        n = sel.numel() if sel is not None else _as_col(cols[key_cols[0]]).t.numel()
    n = int(n)
    cap = n if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    key_descs = (L.TdpCol * len(key_cols))(*[carr[k] for k in key_cols])
    ws_n = L.lib().tdp_groupby_agg_workspace(n, key_descs, len(key_cols), len(aggs), L.STRATEGY[strategy])
    if ws_n == 0:
        raise TdpError(1, "tdp_groupby_agg_workspace")
    ws = workspace(ws_n, dev)
    kout = [torch.empty(max(cap, 1), dtype=_as_col(cols[k]).t.dtype, device=dev) for k in key_cols]
    aout = [torch.empty(max(cap, 1), dtype=torch.int64, device=dev) for _ in aggs]
    ng = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    if sel is not None and nsel is None:
        nsel = torch.tensor([sel.numel()], dtype=torch.int64, device=dev)
    L.call("tdp_groupby_agg", carr, len(cols), pred_array(preds), len(preds), n, _ptr(sel), _ptr(nsel),
           _int_array(key_cols), len(key_cols), agg_array(aggs), len(aggs), L.STRATEGY[strategy],
           _ptr_array(kout), _ptr_array(aout), cap, _ptr(ng), _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"keys": kout, "aggs": aout, "ngroups": ng, "status": status}


# ---------------------------------------------------------------- sort

def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 64, status=None):
    """Stable radix sort of (uint64 key stored in int64, uint32 value stored
    in int32) by the low key_bits bits."""
    _require_cuda(keys, vals)
    dev = keys.device
    n = keys.numel()
    status = new_status(dev) if status is None else status
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    ws_n = L.lib().tdp_sort_pairs_workspace(n, key_bits)
    ws = workspace(ws_n, dev)
    L.call("tdp_sort_pairs", _ptr(keys), _ptr(vals), n, key_bits, _ptr(ko), _ptr(vo), _ptr(ws), ws.numel(),
           _ptr(status), _stream())
    return ko, vo, status


# ---------------------------------------------------------------- join

def join_default_slots(n_keys: int) -> int:
    return int(L.lib().tdp_join_default_slots(int(n_keys)))


def join_build(cols, key_col, payload_col=-1, preds=(), n=None, nslots=None, status=None, table=None, d_n=None):
    carr = col_array(cols)
    dev = _as_col(cols[0]).t.device
    n = _as_col(cols[key_col]).t.numel() if n is None else int(n)
    nslots = join_default_slots(n) if nslots is None else int(nslots)
    status = new_status(dev) if status is None else status
    if table is None:
        table = torch.empty(nslots, dtype=torch.int64, device=dev)
    L.call("tdp_join_build", carr, len(cols), pred_array(preds), len(preds), n, _ptr(d_n), int(key_col),
           int(payload_col),
           L.JOIN_UNIQUE_BUILD, _ptr(table), nslots, _ptr(status), _stream())
    return table, status


def join_probe(table, cols, key_col, preds=(), n=None, sel=None, nsel=None, gather=(), capacity=None,
               rowids=True, payload=True, status=None):
    carr = col_array(cols)
    dev = _as_col(cols[0]).t.device
    if n is None:
        n = sel.numel() if sel is not None else _as_col(cols[key_col]).t.numel()
    n = int(n)
    cap = n if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    orow = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if rowids else None
    opay = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if payload else None
    gout = [torch.empty(max(cap, 1), dtype=_as_col(cols[g]).t.dtype, device=dev) for g in gather]
    count = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    if sel is not None and nsel is None:
        nsel = torch.tensor([sel.numel()], dtype=torch.int64, device=dev)
    ws = workspace(L.lib().tdp_join_probe_workspace(n), dev)
    L.call("tdp_join_probe", _ptr(table), table.numel(), carr, len(cols), pred_array(preds), len(preds), n,
           _ptr(sel), _ptr(nsel), int(key_col), _ptr(orow), _ptr(opay), _int_array(gather), len(gather),
           _ptr_array(gout), cap, _ptr(count), _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"probe_row": orow, "payload": opay, "gathered": gout, "count": count, "status": status}


def join(build_cols, build_key, probe_cols, probe_key, build_payload=-1, build_preds=(), probe_preds=(),
         nslots=None, gather=(), capacity=None, status=None):
    bc = col_array(build_cols)
    pc = col_array(probe_cols)
    dev = _as_col(probe_cols[0]).t.device
    nb = _as_col(build_cols[build_key]).t.numel()
    npr = _as_col(probe_cols[probe_key]).t.numel()
    nslots = join_default_slots(nb) if nslots is None else int(nslots)
    cap = npr if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    orow = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    opay = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    gout = [torch.empty(max(cap, 1), dtype=_as_col(probe_cols[g]).t.dtype, device=dev) for g in gather]
    count = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    ws = workspace(L.lib().tdp_join_workspace(nb, npr, nslots), dev)
    L.call("tdp_join", bc, len(build_cols), pred_array(build_preds), len(build_preds), nb, int(build_key),
           int(build_payload), pc, len(probe_cols), pred_array(probe_preds), len(probe_preds), npr, int(probe_key),
           nslots, _ptr(orow), _ptr(opay), _int_array(gather), len(gather), _ptr_array(gout), cap, _ptr(count),
           _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"probe_row": orow, "payload": opay, "gathered": gout, "count": count, "status": status}


def join_nm(build_cols, build_key, probe_cols, probe_key, build_preds=(), probe_preds=(), capacity=None,
            n_build=None, d_nbuild=None, n_probe=None, d_nprobe=None, status=None):
    """Inner join with repeated build keys: (probe row, build row) pairs in
    probe order, then build-row order.  capacity defaults to the probe row
    count; the true pair count is always written (count)."""
    bc = col_array(build_cols)
    pc = col_array(probe_cols)
    dev = _as_col(probe_cols[0]).t.device
    nb = _as_col(build_cols[build_key]).t.numel() if n_build is None else int(n_build)
    npr = _as_col(probe_cols[probe_key]).t.numel() if n_probe is None else int(n_probe)
    cap = npr if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    op = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    ob = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    ws = workspace(L.lib().tdp_join_nm_workspace(nb, npr), dev)
    L.call("tdp_join_nm", bc, len(build_cols), pred_array(build_preds), len(build_preds), nb, _ptr(d_nbuild),
           int(build_key), pc, len(probe_cols), pred_array(probe_preds), len(probe_preds), npr, _ptr(d_nprobe),
           int(probe_key), _ptr(op), _ptr(ob), cap, _ptr(count), _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"probe_row": op, "build_row": ob, "count": count, "status": status}


def join_probe_agg(table, cols, key_col, lo, hi, aggs, preds=(), n=None, capacity=None, status=None, d_n=None):
    carr = col_array(cols)
    dev = _as_col(cols[0]).t.device
    n = _as_col(cols[key_col]).t.numel() if n is None else int(n)
    D = int(hi) - int(lo) + 1
    cap = D if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    kout = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    aout = [torch.empty(max(cap, 1), dtype=torch.int64, device=dev) for _ in aggs]
    ng = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    ws = workspace(L.lib().tdp_join_probe_agg_workspace(n, D, len(aggs)), dev)
    L.call("tdp_join_probe_agg", _ptr(table), table.numel(), carr, len(cols), pred_array(preds), len(preds), n,
           _ptr(d_n), int(key_col), int(lo), int(hi), agg_array(aggs), len(aggs), _ptr(kout), _ptr_array(aout), cap, _ptr(ng),
           _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"keys": kout, "aggs": aout, "ngroups": ng, "status": status}


def groupjoin(build_cols, build_key, probe_cols, probe_key, lo, hi, aggs, build_preds=(), probe_preds=(),
              n_build=None, d_nbuild=None, n_probe=None, d_nprobe=None, capacity=None, status=None, topk=0,
              topk_agg=0):
    """JOIN build, probe ON key GROUP BY key (build keys unique and bounded by
    [lo, hi]) with aggregates over probe columns.  Returns dict(keys, aggs,
    ngroups, nmatch, status) like groupby_agg; groups in ascending key order.
    topk > 0 adds the fused top-k by aggs[topk_agg] (value desc, key asc):
    top_vals, top_keys, k."""
    bc = col_array(build_cols)
    pc = col_array(probe_cols)
    dev = _as_col(probe_cols[0]).t.device
    nb = _as_col(build_cols[build_key]).t.numel() if n_build is None else int(n_build)
    npr = _as_col(probe_cols[probe_key]).t.numel() if n_probe is None else int(n_probe)
    D = int(hi) - int(lo) + 1
    cap = min(D, max(nb, 0)) if capacity is None else int(capacity)
    status = new_status(dev) if status is None else status
    kout = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    aout = [torch.empty(max(cap, 1), dtype=torch.int64, device=dev) for _ in aggs]
    ng = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    nm = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    topk = int(topk)
    tv = torch.empty(max(topk, 1), dtype=torch.int64, device=dev) if topk else None
    tk = torch.empty(max(topk, 1), dtype=torch.int32, device=dev) if topk else None
    dk = torch.empty(1, dtype=torch.int64, device=dev) if topk else None
    ws_n = L.lib().tdp_groupjoin_workspace(nb, int(lo), int(hi), len(aggs), topk)
    if ws_n == 0:
        raise TdpError(1, "tdp_groupjoin_workspace")
    ws = workspace(ws_n, dev)
    L.call("tdp_groupjoin", bc, len(build_cols), pred_array(build_preds), len(build_preds), nb, _ptr(d_nbuild),
           int(build_key), pc, len(probe_cols), pred_array(probe_preds), len(probe_preds), npr, _ptr(d_nprobe),
           int(probe_key), int(lo), int(hi), agg_array(aggs), len(aggs), _ptr(kout), _ptr_array(aout), cap,
           _ptr(ng), _ptr(nm), topk, int(topk_agg), _ptr(tv), _ptr(tk), _ptr(dk), _ptr(ws), ws.numel(), _ptr(status),
           _stream())
    out = {"keys": [kout], "aggs": aout, "ngroups": ng, "nmatch": nm, "status": status}
    if topk:
        out.update({"top_vals": tv, "top_keys": tk, "k": dk})
    return out


class GroupJoin:
    """The group-join in steps over one workspace: build() once, probe() one
    or more batches of probe rows, finish() for the groups (and top-k).  The
    object owns its workspace and output tensors, so repeated use allocates
    nothing new."""

    def __init__(self, n_build, lo, hi, aggs, topk=0, topk_agg=0, capacity=None, device="cuda"):
        self.n_build, self.lo, self.hi = int(n_build), int(lo), int(hi)
        self.aggs = list(aggs)
        self.topk, self.topk_agg = int(topk), int(topk_agg)
        dev = torch.device(device)
        D = self.hi - self.lo + 1
        self.cap = min(D, max(self.n_build, 0)) if capacity is None else int(capacity)
        n = L.lib().tdp_groupjoin_workspace(self.n_build, self.lo, self.hi, len(self.aggs), self.topk)
        if n == 0:
            raise TdpError(1, "tdp_groupjoin_workspace")
        self.ws = torch.empty(int(n), dtype=torch.uint8, device=dev)
        self.keys = torch.empty(max(self.cap, 1), dtype=torch.int32, device=dev)
        self.out = [torch.empty(max(self.cap, 1), dtype=torch.int64, device=dev) for _ in self.aggs]
        self.ngroups = torch.empty(1, dtype=torch.int64, device=dev)
        self.nmatch = torch.empty(1, dtype=torch.int64, device=dev)
        self.top_vals = torch.empty(max(self.topk, 1), dtype=torch.int64, device=dev)
        self.top_keys = torch.empty(max(self.topk, 1), dtype=torch.int32, device=dev)
        self.k = torch.empty(1, dtype=torch.int64, device=dev)
        self._agg_arr = agg_array(self.aggs)

    def build(self, cols, key_col, preds=(), d_n=None, status=None):
        L.call("tdp_groupjoin_build", col_array(cols), len(cols), pred_array(preds), len(preds), self.n_build,
               _ptr(d_n), int(key_col), self.lo, self.hi, self._agg_arr, len(self.aggs), self.topk, _ptr(self.ws),
               self.ws.numel(), _ptr(status), _stream())

    def probe(self, cols, key_col, preds=(), n=None, d_n=None, status=None):
        n = _as_col(cols[key_col]).t.numel() if n is None else int(n)
        L.call("tdp_groupjoin_probe", col_array(cols), len(cols), pred_array(preds), len(preds), n, _ptr(d_n),
               int(key_col), self.n_build, self.lo, self.hi, self._agg_arr, len(self.aggs), self.topk,
               _ptr(self.ws), self.ws.numel(), _ptr(status), _stream())

    def finish(self, status=None):
        tk = self.topk > 0
        L.call("tdp_groupjoin_finish", self.n_build, self.lo, self.hi, self._agg_arr, len(self.aggs),
               _ptr(self.keys), _ptr_array(self.out), self.cap, _ptr(self.ngroups), _ptr(self.nmatch), self.topk,
               self.topk_agg, _ptr(self.top_vals) if tk else None, _ptr(self.top_keys) if tk else None,
               _ptr(self.k) if tk else None, _ptr(self.ws), self.ws.numel(), _ptr(status), _stream())
        out = {"keys": [self.keys], "aggs": self.out, "ngroups": self.ngroups, "nmatch": self.nmatch}
        if tk:
            out.update({"top_vals": self.top_vals, "top_keys": self.top_keys, "k": self.k})
        return out


def dict_encode(offsets, data, max_len=32, dict_cap=None, bytes_cap=None, status=None):
    """Order-preserving dictionary codes of a string column (offsets int32
    [n+1], data uint8).  Returns dict(codes int32[n], dict_offsets, dict_bytes,
    ndict, nbytes (device int64[1] each), status)."""
    _require_cuda(offsets, data)
    dev = offsets.device
    n = offsets.numel() - 1
    dict_cap = n if dict_cap is None else int(dict_cap)
    bytes_cap = data.numel() if bytes_cap is None else int(bytes_cap)
    status = new_status(dev) if status is None else status
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    doff = torch.empty(dict_cap + 1, dtype=torch.int32, device=dev)
    dbytes = torch.empty(max(bytes_cap, 1), dtype=torch.uint8, device=dev)
    nd = torch.empty(1, dtype=torch.int64, device=dev)
    nbt = torch.empty(1, dtype=torch.int64, device=dev)
    ws_n = L.lib().tdp_dict_encode_workspace(n, int(max_len))
    if ws_n == 0:
        raise TdpError(1, "tdp_dict_encode_workspace")
    ws = workspace(ws_n, dev)
    L.call("tdp_dict_encode", _ptr(offsets), _ptr(data), n, int(max_len), _ptr(codes), _ptr(doff), _ptr(dbytes),
           dict_cap, bytes_cap, _ptr(nd), _ptr(nbt), _ptr(ws), ws.numel(), _ptr(status), _stream())
    return {"codes": codes, "dict_offsets": doff, "dict_bytes": dbytes, "ndict": nd, "nbytes": nbt,
            "status": status}


# ---------------------------------------------------------------- top-k

def topk(vals, keys, k, d_n=None, status=None):
    _require_cuda(vals, keys)
    dev = vals.device
    n = vals.numel()
    status = new_status(dev) if status is None else status
    ov = torch.empty(k, dtype=torch.int64, device=dev)
    okk = torch.empty(k, dtype=torch.int32, device=dev)
    dk = torch.empty(1, dtype=torch.int64, device=dev)  # written by the call
    ws = workspace(L.lib().tdp_topk_workspace(n, k), dev)
    L.call("tdp_topk", _ptr(vals), _ptr(keys), n, _ptr(d_n), int(k), _ptr(ov), _ptr(okk), _ptr(dk), _ptr(ws),
           ws.numel(), _ptr(status), _stream())
    return ov, okk, dk


# ---------------------------------------------------------- soft operators

def _soft_ws(n, G, dev):
    return workspace(L.lib().tdp_soft_workspace(n, G), dev)


def soft_filter_fwd(x, gid, theta, tau):
    _require_cuda(x, gid, theta)
    mask = torch.empty_like(x)
    L.call("tdp_soft_filter_fwd", _ptr(x), _ptr(gid), _ptr(theta), float(tau), x.numel(), _ptr(mask), _stream())
    return mask


def soft_filter_bwd(x, gid, theta, tau, grad_mask, need_x=True):
    _require_cuda(x, gid, theta, grad_mask)
    G = theta.numel()
    gth = torch.empty_like(theta)
    gx = torch.empty_like(x) if need_x else None
    ws = _soft_ws(x.numel(), G, x.device)
    L.call("tdp_soft_filter_bwd", _ptr(x), _ptr(gid), _ptr(theta), float(tau), x.numel(), G, _ptr(grad_mask),
           _ptr(gx), _ptr(gth), _ptr(ws), ws.numel(), _stream())
    return gth, gx


def soft_agg_fwd(x, v, gid, theta, tau):
    _require_cuda(x, v, gid, theta)
    G = theta.numel()
    S = torch.empty(G, dtype=torch.float32, device=x.device)
    Cn = torch.empty(G, dtype=torch.float32, device=x.device)
    ws = _soft_ws(x.numel(), G, x.device)
    L.call("tdp_soft_agg_fwd", _ptr(x), _ptr(v), _ptr(gid), _ptr(theta), float(tau), x.numel(), G, _ptr(S),
           _ptr(Cn), _ptr(ws), ws.numel(), _stream())
    return S, Cn


def soft_agg_bwd(x, v, gid, theta, tau, gsum, gcnt, need_v=False, need_x=False):
    _require_cuda(x, v, gid, theta, gsum, gcnt)
    G = theta.numel()
    gth = torch.empty_like(theta)
    gv = torch.empty_like(v) if need_v else None
    gx = torch.empty_like(x) if need_x else None
    ws = _soft_ws(x.numel(), G, x.device)
    L.call("tdp_soft_agg_bwd", _ptr(x), _ptr(v), _ptr(gid), _ptr(theta), float(tau), x.numel(), G, _ptr(gsum),
           _ptr(gcnt), _ptr(gth), _ptr(gv), _ptr(gx), _ptr(ws), ws.numel(), _stream())
    return gth, gv, gx
