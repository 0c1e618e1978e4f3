"""GPU parity of the soft (trainable) operators against the fp64 oracle and
float64 finite differences.  Tolerance per output element:
|gpu - ref| <= 1e-5 * max(|ref|, 1e-3 * max_j |ref_j|)."""
import numpy as np
import pytest
import torch

import gen
from oracle import soft
from paper_2211_02753_b300 import autograd as A
from paper_2211_02753_b300 import ops

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TAU = float(np.float32(0.1))  # the kernels take tau as fp32; the oracle gets the same value
RTOL = 1e-5


def close(got, ref, rtol=RTOL):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 1e-3 * np.abs(ref).max() if ref.size else 0.0
    tol = rtol * np.maximum(np.abs(ref), floor)
    bad = np.abs(got - ref) > tol
    return not bad.any(), (np.abs(got - ref) / np.maximum(np.abs(ref), floor + 1e-300)).max() if ref.size else 0


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# empty input, one row, ragged tails, the maximum group count (4096), the 10M-row workload
@pytest.mark.parametrize("n,G", [(0, 5), (1, 1), (4099, 7), (50001, 4096), (100003, 1024), (10_000_000, 1024)])
def test_soft_agg_fwd_bwd(n, G):
    d = gen.soft_table(n, G, gen.BASE_SEED + 3)
    r = np.random.default_rng(n)
    theta = (r.standard_normal(G) * 0.5).astype(np.float32)
    gS = r.standard_normal(G).astype(np.float32)
    gC = r.standard_normal(G).astype(np.float32)
    x, v, gid, th = cu(d["x"]), cu(d["v"]), cu(d["gid"]), cu(theta)
    S, C = ops.soft_agg_fwd(x, v, gid, th, TAU)
    rS, rC = soft.soft_agg_fwd(d["x"], d["v"], d["gid"], theta, TAU, G)
    ok, err = close(S.cpu().numpy(), rS)
    assert ok, err
    ok, err = close(C.cpu().numpy(), rC)
    assert ok, err
    gth, gv, gx = ops.soft_agg_bwd(x, v, gid, th, TAU, cu(gS), cu(gC), need_v=True, need_x=True)
    rth, rv, rx = soft.soft_agg_bwd(d["x"], d["v"], d["gid"], theta, TAU, G, gS, gC)
    ok, err = close(gth.cpu().numpy(), rth)
    assert ok, err
    idx = np.random.default_rng(1).choice(n, size=min(n, 100000), replace=False)
    ok, err = close(gv.cpu().numpy()[idx], rv[idx])
    assert ok, err
    ok, err = close(gx.cpu().numpy()[idx], rx[idx])
    assert ok, err


def test_soft_filter_fwd_bwd():
    n, G = 300001, 64
    d = gen.soft_table(n, G, 77)
    r = np.random.default_rng(2)
    theta = r.standard_normal(G).astype(np.float32)
    gm = r.standard_normal(n).astype(np.float32)
    x, gid, th = cu(d["x"]), cu(d["gid"]), cu(theta)
    m = ops.soft_filter_fwd(x, gid, th, TAU)
    rm = soft.soft_filter_fwd(d["x"], d["gid"], theta, TAU)
    ok, err = close(m.cpu().numpy(), rm)
    assert ok, err
    gth, gx = ops.soft_filter_bwd(x, gid, th, TAU, cu(gm))
    rth, rx = soft.soft_filter_bwd(d["x"], d["gid"], theta, TAU, G, gm)
    ok, err = close(gth.cpu().numpy(), rth)
    assert ok, err
    ok, err = close(gx.cpu().numpy(), rx)
    assert ok, err


def test_soft_mask_half_at_threshold_and_hard_limit():
    x = cu(np.array([0.3, -1.0, 2.0], np.float32))
    gid = cu(np.array([0, 1, 2], np.int32))
    th = cu(np.array([0.3, -1.0, 1.0], np.float32))
    m = ops.soft_filter_fwd(x, gid, th, TAU).cpu().numpy()
    assert m[0] == 0.5 and m[1] == 0.5 and m[2] > 0.9999
    m = ops.soft_filter_fwd(x, gid, th, 1e-6).cpu().numpy()
    assert m[2] == 1.0


def test_gpu_gradient_vs_finite_differences():
    """theta.grad from the hand-written adjoint vs float64 central differences
    of L = a.S + b.C computed by the oracle."""
    n, G = 20000, 16
    d = gen.soft_table(n, G, 5)
    r = np.random.default_rng(5)
    theta = (r.standard_normal(G) * 0.3).astype(np.float32)
    a, b = r.standard_normal(G), r.standard_normal(G)
    th = cu(theta).requires_grad_(True)
    S, C = A.SoftAgg.apply(cu(d["x"]), cu(d["v"]), cu(d["gid"]), th, TAU)
    L = (S.double() * cu(a)).sum() + (C.double() * cu(b)).sum()
    L.backward()
    g = th.grad.cpu().numpy()
    h = 1e-6
    for j in range(G):
        e = np.zeros(G)
        e[j] = h
        Sp, Cp = soft.soft_agg_fwd(d["x"], d["v"], d["gid"], theta.astype(np.float64) + e, TAU, G)
        Sm, Cm = soft.soft_agg_fwd(d["x"], d["v"], d["gid"], theta.astype(np.float64) - e, TAU, G)
        fd = ((a @ Sp + b @ Cp) - (a @ Sm + b @ Cm)) / (2 * h)
        assert abs(g[j] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(g).max()), (j, g[j], fd)


def test_autograd_filter_chain_matches_oracle():
    n, G = 50000, 32
    d = gen.soft_table(n, G, 8)
    theta = np.linspace(-1, 1, G).astype(np.float32)
    gm = np.random.default_rng(8).standard_normal(n).astype(np.float32)
    th = cu(theta).requires_grad_(True)
    x = cu(d["x"]).requires_grad_(True)
    m = A.SoftFilter.apply(x, cu(d["gid"]), th, TAU)
    m.backward(cu(gm))
    rth, rx = soft.soft_filter_bwd(d["x"], d["gid"], theta, TAU, G, gm)
    ok, err = close(th.grad.cpu().numpy(), rth)
    assert ok, err
    ok, err = close(x.grad.cpu().numpy(), rx)
    assert ok, err


def test_determinism_across_runs():
    n, G = 1_000_000, 1024
    d = gen.soft_table(n, G, 3)
    x, v, gid = cu(d["x"]), cu(d["v"]), cu(d["gid"])
    th = torch.zeros(G, device=DEV)
    outs = [torch.cat(ops.soft_agg_fwd(x, v, gid, th, TAU)).cpu().numpy() for _ in range(3)]
    for o in outs[1:]:
        ok, err = close(o, outs[0], rtol=1e-6)
        assert ok, err
