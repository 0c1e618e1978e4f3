"""GPU parity of the soft ORDER BY ... LIMIT k against the float64 oracle.

Tolerances, from the arithmetic.  A logistic term is rcp(1 + 2^z) with
z = x_i c - x_j c, c = log2(e) / tau, each product rounded to fp32: for
|x c| <= 2^8 the rounding moves z by at most 2^-15, the term by at most
ln2 / 4 * 2^-15 < 5.3e-6; the two approximate special functions add about
2^-21 relative; an fp32 partial of 32 terms in [0, 1] adds at most
31 * 2^-24 per term, and the partials are added with compensation.  So a
rank over n rows is off by |dr| <= 8e-6 n + 1e-5.  The membership moves by at most
m (1 - m) / tau_r times that, a group sum by the sum of |v| times the
membership bound, and dx_i by 3e-5 of (|A_i| + |dr_i| B_i) / tau, with
A_i = sum_j w_ij |dr_j| and B_i = sum_j w_ij (the terms of the two sums whose
difference is dx_i).  Exact ranks are integers: bit-exact.
"""
import numpy as np
import pytest
import torch

import gen
from oracle import soft as SO
from oracle import softsort as O
from paper_2211_02753_b300 import softsort as ss

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _groups(sizes, seed, ties=False):
    r = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = r.standard_normal(offs[-1]).astype(np.float32)
    if ties:
        x = np.round(x * 4).astype(np.float32) / 4
    v = r.uniform(0, 100, offs[-1]).astype(np.float32)
    return x, v, offs


LAYOUTS = [
    ((1,), False),
    ((2, 7, 33, 300), True),             # ties, a 300-row group over two row tiles
    ((0, 5, 0, 2500, 1), True),           # empty groups, a group over two staged chunks
    ((256, 257, 511, 512, 513), False),  # tile edges
]


@pytest.mark.parametrize("sizes,ties", LAYOUTS)
def test_exact_ranks_and_sums(sizes, ties):
    x, v, offs = _groups(sizes, sum(sizes), ties)
    for k in (1, 3, 1000):
        rank, S = ss.exact_topk(dev(x), dev(v), dev(offs), k)
        assert np.array_equal(rank.cpu().numpy(), O.exact_rank(x, offs))
        assert np.allclose(S.cpu().numpy(), O.exact_topk_sum(x, v, offs, k), rtol=1e-12, atol=0)


def _rank_tol(offs, n_rows_of):
    sizes = np.diff(offs)
    return np.repeat(8e-6 * sizes + 1e-5, sizes)


@pytest.mark.parametrize("sizes,ties", LAYOUTS)
@pytest.mark.parametrize("tau,tau_r,k", [(0.1, 0.5, 3), (1.0, 2.0, 10)])
def test_soft_forward(sizes, ties, tau, tau_r, k):
    x, v, offs = _groups(sizes, 7 + sum(sizes), ties)
    rank, mask, S = ss.soft_topk_fwd(dev(x), dev(v), dev(offs), k, tau, tau_r)
    r_ref, m_ref, S_ref = O.soft_topk_fwd(x, v, offs, k, tau, tau_r)
    tol_r = _rank_tol(offs, None)
    got_r = rank.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got_r - r_ref) <= tol_r)
    tol_m = m_ref * (1 - m_ref) / tau_r * tol_r + 1e-6
    assert np.all(np.abs(mask.cpu().numpy() - m_ref) <= tol_m)
    for g, (a, b) in enumerate(zip(offs[:-1], offs[1:])):
        bound = float(np.sum(np.abs(v[a:b]) * tol_m[a:b])) + 1e-6 * abs(S_ref[g]) + 1e-6
        assert abs(float(S[g].item()) - S_ref[g]) <= bound
        n = b - a
        assert abs(got_r[a:b].sum() - n * (n + 1) / 2) <= tol_r[a:b].sum() + 1e-6  # the rank-sum invariant


@pytest.mark.parametrize("sizes,ties", LAYOUTS)
def test_soft_backward(sizes, ties):
    x, v, offs = _groups(sizes, 11 + sum(sizes), ties)
    k, tau, tau_r = 3, 0.2, 0.5
    r = np.random.default_rng(3)
    dS = r.standard_normal(len(offs) - 1).astype(np.float32)
    dm = r.standard_normal(x.shape[0]).astype(np.float32)
    dr = r.standard_normal(x.shape[0]).astype(np.float32)
    _, m_ref, _ = O.soft_topk_fwd(x, v, offs, k, tau, tau_r)
    m32 = m_ref.astype(np.float32)  # the same membership on both sides
    dx, dv = ss.soft_topk_bwd(dev(x), dev(v), dev(offs), k, tau, tau_r, dev(m32), dsum=dev(dS), dmask=dev(dm),
                              drank=dev(dr))
    rdx, rdv = O.soft_topk_bwd(x, v, offs, k, tau, tau_r, m32, dS=dS, dm=dm, dr=dr)
    assert np.allclose(dv.cpu().numpy(), rdv, rtol=1e-6, atol=1e-6)
    # the tolerance of dx: 3e-5 of the two sums whose difference it is
    m = m32.astype(np.float64)
    drv = -(np.repeat(dS, np.diff(offs)) * v + dm) * m * (1 - m) / tau_r + dr
    got = dx.cpu().numpy()
    for a, b in zip(offs[:-1], offs[1:]):
        xs = x[a:b].astype(np.float64)
        sg = SO.sigmoid((xs[None, :] - xs[:, None]) / tau)
        w = sg * (1 - sg)
        bound = 3e-5 * (w @ np.abs(drv[a:b]) + np.abs(drv[a:b]) * w.sum(axis=1)) / tau + 1e-6
        assert np.all(np.abs(got[a:b] - rdx[a:b]) <= bound)


def test_autograd_soft_topk_sum():
    x, v, offs = _groups((40, 90, 7), 5)
    gx, gv = dev(x).requires_grad_(True), dev(v).requires_grad_(True)
    S = ss.SoftTopKSum.apply(gx, gv, dev(offs), 5, 0.3, 0.5, 90)
    w = torch.tensor([1.0, -2.0, 0.5], device=DEV)
    (S * w).sum().backward()
    _, m, _ = O.soft_topk_fwd(x, v, offs, 5, 0.3, 0.5)
    rdx, rdv = O.soft_topk_bwd(x, v, offs, 5, 0.3, 0.5, m, dS=w.cpu().numpy().astype(np.float64))
    assert np.allclose(gv.grad.cpu().numpy(), rdv, rtol=1e-5, atol=1e-5)
    assert np.linalg.norm(gx.grad.cpu().numpy() - rdx) <= 1e-4 * np.linalg.norm(rdx)


def test_oversized_and_malformed_groups_set_capacity():
    x, v, offs = _groups((10, 20, 5), 9)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    rank = torch.full((35,), -7, dtype=torch.int32, device=DEV)
    # max_group 12: the 20-row group is skipped
    r, S = ss.exact_topk(dev(x), dev(v), dev(offs), 3, max_group=12, status=st)
    assert int(st.item()) == 4
    rr = r.cpu().numpy()
    er = O.exact_rank(x, offs)
    assert np.array_equal(rr[:10], er[:10]) and np.array_equal(rr[30:], er[30:])
    assert float(S[1].item()) == 0.0
    st.zero_()
    bad = np.array([0, 20, 10, 35], np.int64)  # out of order
    ss.exact_topk(dev(x), dev(v), dev(bad), 3, max_group=40, status=st)
    assert int(st.item()) == 4
    del rank


def test_workload_size_sampled_groups():
    """The benchmark's workload (1000 groups of 500..1500 rows, 1M rows):
    forward and backward of the soft top-10 sum, 25 sampled groups against
    the oracle, and the exact operator everywhere by the rank-sum identity
    and against the oracle on the same sample."""
    d = gen.ranked_groups(1000, 1000, gen.BASE_SEED + 11)
    x, v, offs = d["x"], d["v"], d["offsets"]
    k, tau, tau_r = 10, 0.05, 0.5
    gx, gv, go = dev(x), dev(v), dev(offs)
    rank, mask, S = ss.soft_topk_fwd(gx, gv, go, k, tau, tau_r, max_group=1500)
    dS = torch.ones(1000, device=DEV)
    dx, dv = ss.soft_topk_bwd(gx, gv, go, k, tau, tau_r, mask, dsum=dS, max_group=1500)
    er, eS = ss.exact_topk(gx, gv, go, k, max_group=1500)
    rank, mask, S, dx, er, eS = (t.cpu().numpy() for t in (rank, mask, S, dx, er, eS))
    sizes = np.diff(offs)
    assert np.array_equal(np.add.reduceat(er.astype(np.int64), offs[:-1]), sizes * (sizes + 1) // 2)
    r0 = np.random.default_rng(2)
    for g in r0.choice(1000, 25, replace=False):
        a, b = int(offs[g]), int(offs[g + 1])
        lo = np.array([0, b - a])
        xs, vs = x[a:b], v[a:b]
        rr, mm, SS = O.soft_topk_fwd(xs, vs, lo, k, tau, tau_r)
        tol_r = 8e-6 * (b - a) + 1e-5
        assert np.all(np.abs(rank[a:b] - rr) <= tol_r)
        tol_m = mm * (1 - mm) / tau_r * tol_r + 1e-6
        assert abs(S[g] - SS[0]) <= np.sum(vs * tol_m) + 1e-6 * abs(SS[0]) + 1e-6
        rdx, _ = O.soft_topk_bwd(xs, vs, lo, k, tau, tau_r, mask[a:b], dS=np.ones(1))
        assert np.linalg.norm(dx[a:b] - rdx) <= 1e-3 * np.linalg.norm(rdx) + 1e-6
        assert np.array_equal(er[a:b], O.exact_rank(xs, lo))
        assert np.allclose(eS[g], O.exact_topk_sum(xs, vs, lo, k)[0], rtol=1e-12)
