"""tdp_soft_agg_fwd_noalloc: the soft aggregation forward for callers that
cannot allocate device memory (its scratch is a fixed array inside the
library).  Checked through the C ABI against tdp_soft_agg_fwd, the entry
point with a caller workspace, and against the float64 oracle, on calls in a
row (a later call must not see anything left behind by an earlier one), with
the tolerance the soft tests use: |a - b| <= 1e-5 * max(|b|, 1e-3 * max|b|).

The first call has 10M rows, more than the 256 blocks of the fixed scratch
hold at the normal grid (about 4.2M rows), so it takes the capped grid with
longer chunks; the calls after it are smaller and fill fewer blocks of the
array than the first one left behind.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import gen
from oracle import soft as O
from paper_2211_02753_b300 import _lib as L

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TAU = float(np.float32(0.1))


def _p(t):
    return C.c_void_p(t.data_ptr())


def _close(a, b, rtol=1e-5):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    floor = 1e-3 * np.abs(b).max()
    return bool(np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(b), floor)))


def _inputs(n, G, seed):
    d = gen.soft_table(n, G, seed)
    theta = (np.random.default_rng(seed).standard_normal(G) * 0.5).astype(np.float32)
    return [torch.from_numpy(a).to(DEV) for a in (d["x"], d["v"], d["gid"], theta)]


def _with_workspace(x, v, gid, th, G):
    lib = L.lib()
    ws = torch.empty(int(lib.tdp_soft_workspace(x.numel(), G)), dtype=torch.uint8, device=DEV)
    S = torch.empty(G, dtype=torch.float32, device=DEV)
    Cn = torch.empty(G, dtype=torch.float32, device=DEV)
    st = lib.tdp_soft_agg_fwd(_p(x), _p(v), _p(gid), _p(th), TAU, x.numel(), G, _p(S), _p(Cn), _p(ws), ws.numel(),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return S.cpu().numpy(), Cn.cpu().numpy()


def _no_alloc(x, v, gid, th, G, S, Cn):
    st = L.lib().tdp_soft_agg_fwd_noalloc(_p(x), _p(v), _p(gid), _p(th), TAU, x.numel(), G, _p(S), _p(Cn),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


def test_no_alloc_matches_workspace_entry_point_twice():
    G = 1024
    S = torch.empty(G, dtype=torch.float32, device=DEV)
    Cn = torch.empty(G, dtype=torch.float32, device=DEV)
    # calls in a row on different inputs and sizes: the capped grid first,
    # then the normal grid with fewer blocks, then the capped grid again
    for n, seed in ((10_000_000, 10), (3_000_001, 11), (777_777, 12), (4_500_000, 14)):
        x, v, gid, th = _inputs(n, G, seed)
        rS, rC = _with_workspace(x, v, gid, th, G)
        assert _no_alloc(x, v, gid, th, G, S, Cn) == 0
        gS, gC = S.cpu().numpy(), Cn.cpu().numpy()
        assert _close(gS, rS) and _close(gC, rC)
        oS, oC = O.soft_agg_fwd(x.cpu().numpy(), v.cpu().numpy(), gid.cpu().numpy(), th.cpu().numpy(), TAU, G)
        assert _close(gS, oS) and _close(gC, oC)


def test_no_alloc_rejects_too_many_groups():
    G = 1025
    x, v, gid, th = _inputs(1000, G, 13)
    S = torch.empty(G, dtype=torch.float32, device=DEV)
    Cn = torch.empty(G, dtype=torch.float32, device=DEV)
    assert _no_alloc(x, v, gid, th, G, S, Cn) == 3  # TDP_ERR_WORKSPACE_TOO_SMALL
