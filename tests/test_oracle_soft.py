"""Pins for the fp64 soft-operator oracle (Sec. 4: logistic relaxation of a
filter predicate, COUNT on probability-encoded data from + and x only,
soft_groupby, exact operators swapped in at inference).

Checked against closed forms (m = 1/2 at x = theta), the tau -> 0 limit
(the hard filter), central finite differences in float64, and the one-hot
special case (soft COUNT equals the exact COUNT).
"""
import numpy as np
import pytest

from oracle import soft

TAU = 0.1


def _rows(seed, n, G):
    r = np.random.default_rng(seed)
    x = r.standard_normal(n).astype(np.float32)
    v = (r.random(n) * 100).astype(np.float32)
    gid = r.integers(0, G, n).astype(np.int32)
    theta = (r.standard_normal(G) * 0.3).astype(np.float32)
    return x, v, gid, theta


def test_mask_half_at_threshold_and_slope():
    th = np.array([0.25, -1.0], np.float32)
    x = th.copy()
    m = soft.soft_mask(x, np.array([0, 1]), th, TAU)
    assert np.all(m == 0.5)
    # dm/dtheta = -m(1-m)/tau = -1/(4 tau) at z = 0
    h = 1e-6
    fd = (soft.soft_mask(x, [0, 1], th.astype(np.float64) + h, TAU)
          - soft.soft_mask(x, [0, 1], th.astype(np.float64) - h, TAU)) / (2 * h)
    assert np.allclose(fd, -1.0 / (4 * TAU), rtol=1e-7)
    assert np.allclose(soft.dmask_dz(x, [0, 1], th, TAU), 0.25)


def test_sigmoid_extremes_are_finite():
    z = np.array([-800.0, -40.0, 0.0, 40.0, 800.0])
    s = soft.sigmoid(z)
    assert np.all(np.isfinite(s)) and s[0] == 0.0 and s[-1] == 1.0 and s[2] == 0.5


def test_tau_to_zero_is_hard_filter():
    x, v, gid, theta = _rows(1, 5000, 16)
    keep = np.abs(x.astype(np.float64) - theta[gid]) > 1e-3
    x, v, gid = x[keep], v[keep], gid[keep]
    S, C = soft.soft_agg_fwd(x, v, gid, theta, 1e-6, 16)
    Sh, Ch = soft.hard_agg(x, v, gid, theta, 16)
    assert np.allclose(S, Sh, rtol=0, atol=1e-9 * np.abs(Sh).max())
    assert np.array_equal(np.rint(C), Ch)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_agg_theta_gradient_vs_finite_differences(seed):
    G = 8
    x, v, gid, theta = _rows(seed, 3000, G)
    r = np.random.default_rng(1000 + seed)
    a, b = r.standard_normal(G), r.standard_normal(G)

    def L(th):
        S, C = soft.soft_agg_fwd(x, v, gid, th, TAU, G)
        return float(a @ S + b @ C)

    dth, dv, dx = soft.soft_agg_bwd(x, v, gid, theta, TAU, G, a, b)
    h = 1e-6
    th64 = theta.astype(np.float64)
    for g in range(G):
        e = np.zeros(G)
        e[g] = h
        fd = (L(th64 + e) - L(th64 - e)) / (2 * h)
        assert abs(fd - dth[g]) <= 1e-7 * max(abs(dth[g]), 1e-3 * np.abs(dth).max()) + 1e-9, (g, fd, dth[g])


def test_agg_row_gradients_vs_finite_differences():
    G = 4
    x, v, gid, theta = _rows(7, 200, G)
    r = np.random.default_rng(7)
    a, b = r.standard_normal(G), r.standard_normal(G)
    x64, v64 = x.astype(np.float64), v.astype(np.float64)

    def L(xx, vv):
        S, C = soft.soft_agg_fwd(xx, vv, gid, theta, TAU, G)
        return float(a @ S + b @ C)

    _, dv, dx = soft.soft_agg_bwd(x, v, gid, theta, TAU, G, a, b)
    h = 1e-6
    for i in range(0, 200, 17):
        e = np.zeros(200)
        e[i] = h
        fdx = (L(x64 + e, v64) - L(x64 - e, v64)) / (2 * h)
        fdv = (L(x64, v64 + e) - L(x64, v64 - e)) / (2 * h)
        assert abs(fdx - dx[i]) <= 1e-6 * max(1.0, abs(dx[i]))
        assert abs(fdv - dv[i]) <= 1e-6 * max(1.0, abs(dv[i]))


def test_filter_bwd_vs_finite_differences():
    G = 5
    x, _, gid, theta = _rows(9, 400, G)
    gm = np.random.default_rng(9).standard_normal(400)

    def L(th):
        return float(gm @ soft.soft_filter_fwd(x, gid, th, TAU))

    dth, dx = soft.soft_filter_bwd(x, gid, theta, TAU, G, gm)
    h = 1e-6
    for g in range(G):
        e = np.zeros(G)
        e[g] = h
        fd = (L(theta.astype(np.float64) + e) - L(theta.astype(np.float64) - e)) / (2 * h)
        assert abs(fd - dth[g]) <= 1e-7 * max(1.0, abs(dth[g]))
    # dx: central differences of the same loss in every row's x (the loss is a
    # sum over rows, so one perturbation per row moves only that row's term)
    x64 = x.astype(np.float64)

    def Lx(xx):
        return float(gm @ soft.soft_filter_fwd(xx, gid, theta, TAU))

    assert dx.shape == x.shape
    for i in range(0, 400, 7):
        e = np.zeros(400)
        e[i] = h
        fd = (Lx(x64 + e) - Lx(x64 - e)) / (2 * h)
        assert abs(fd - dx[i]) <= 1e-6 * max(1.0, abs(dx[i]))
    # sign and scale of the adjoint: at x = theta the mask slope is 1/(4 tau)
    xm = theta[gid].astype(np.float32)
    _, dxm = soft.soft_filter_bwd(xm, gid, theta, TAU, G, np.ones(400))
    assert np.allclose(dxm, 0.25 / TAU, rtol=1e-12)


def test_onehot_pe_count_is_exact():
    r = np.random.default_rng(3)
    labels = r.integers(0, 10, (32, 4, 4))
    P = np.eye(10)[labels.reshape(-1)].astype(np.float32)
    cnt, rsum = soft.pe_groupby_fwd(P)
    ecnt, ersum = soft.exact_groupby(labels)
    assert np.array_equal(cnt, ecnt) and np.array_equal(rsum, ersum)
    # hand check on one grid: labels row-major
    lab = np.arange(16).reshape(1, 4, 4) % 10
    c1, r1 = soft.exact_groupby(lab)
    assert c1[0].tolist() == [2, 2, 2, 2, 2, 2, 1, 1, 1, 1]
    assert r1[0].tolist() == [0 + 1 + 2 + 3, 4 + 5 + 6 + 7, 8 + 9 + 0 + 1, 2 + 3 + 4 + 5]


def test_pe_groupby_adjoint_identity():
    """pe_groupby is linear in P; its backward must be the exact adjoint."""
    r = np.random.default_rng(5)
    P = r.random((3 * 16, 10))
    dcnt, drsum = r.standard_normal((3, 10)), r.standard_normal((3, 4))
    cnt, rsum = soft.pe_groupby_fwd(P)
    dP = soft.pe_groupby_bwd(dcnt, drsum)
    assert np.isclose((dP * P).sum(), (dcnt * cnt).sum() + (drsum * rsum).sum(), rtol=1e-12)


def test_pe_groupby2_pins():
    """The two-attribute soft COUNT (Digit x Size): per grid it is the matrix
    product Pa^T Pb of the grid's cells (a library routine), one-hot inputs
    give the exact pair counts bitwise, and the backward is the exact
    adjoint of the bilinear map in each argument."""
    r = np.random.default_rng(21)
    n, cells = 5, 16
    Pa = r.random((n * cells, 10))
    Pb = r.random((n * cells, 2))
    cnt = soft.pe_groupby2_fwd(Pa, Pb)
    for g in range(n):
        A = Pa[g * cells:(g + 1) * cells]
        B = Pb[g * cells:(g + 1) * cells]
        assert np.allclose(cnt[g], A.T @ B, rtol=1e-12)
    dig = r.integers(0, 10, (n, 4, 4))
    siz = r.integers(0, 2, (n, 4, 4))
    oh = soft.pe_groupby2_fwd(np.eye(10)[dig.reshape(-1)], np.eye(2)[siz.reshape(-1)])
    assert np.array_equal(oh, soft.exact_groupby2(dig, siz).astype(np.float64))
    assert soft.exact_groupby2(dig, siz).sum() == n * 16
    d = r.standard_normal((n, 10, 2))
    dA, dB = soft.pe_groupby2_bwd(d, Pa, Pb)
    lhs = (d * cnt).sum()
    assert np.isclose((dA * Pa).sum(), lhs, rtol=1e-12) and np.isclose((dB * Pb).sum(), lhs, rtol=1e-12)
