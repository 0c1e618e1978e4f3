"""Pins of the soft ORDER BY / top-k oracle to brute-force sorting, the
invariants of the logistic relaxation, its limits and finite differences."""
import numpy as np

from oracle import softsort as O


def _case(seed, sizes=(1, 2, 7, 40, 100)):
    r = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    x = r.standard_normal(offs[-1])
    v = r.uniform(0, 100, offs[-1])
    return x, v, offs


def test_exact_rank_is_the_position_in_a_stable_descending_sort():
    x, v, offs = _case(1)
    x = np.round(x, 1)  # ties
    r = O.exact_rank(x, offs)
    for a, b in zip(offs[:-1], offs[1:]):
        order = sorted(range(a, b), key=lambda i: (-x[i], i))  # brute force: stable sort, descending
        for pos, i in enumerate(order):
            assert r[i] == pos + 1
    k = 3
    S = O.exact_topk_sum(x, v, offs, k)
    for g, (a, b) in enumerate(zip(offs[:-1], offs[1:])):
        order = sorted(range(a, b), key=lambda i: (-x[i], i))
        assert np.isclose(S[g], sum(v[i] for i in order[:k]), rtol=1e-12)


def test_soft_rank_invariant_and_limits():
    x, v, offs = _case(2)
    r = O.soft_rank(x, offs, 0.3)
    for a, b in zip(offs[:-1], offs[1:]):
        n = b - a
        # sigma(z) + sigma(-z) = 1: the soft ranks of a group sum to n (n + 1) / 2
        assert np.isclose(r[a:b].sum(), n * (n + 1) / 2, rtol=1e-12)
        assert np.all(r[a:b] >= 1) and np.all(r[a:b] <= n)
    # tau -> 0 on distinct values: the exact descending rank
    assert np.allclose(O.soft_rank(x, offs, 1e-9), O.exact_rank(x, offs), atol=1e-9)
    # a tie contributes one half to each of the tied rows
    r2 = O.soft_rank(np.array([1.0, 1.0, 3.0]), [0, 3], 1e-6)
    assert np.allclose(r2, [2.5, 2.5, 1.0])
    # a large tau flattens every comparison to one half
    assert np.allclose(O.soft_rank(x[:40], [0, 40], 1e9), 1 + 39 / 2)


def test_membership_limit_is_the_exact_top_k_sum():
    x, v, offs = _case(3)
    for k in (1, 5, 200):
        _, m, S = O.soft_topk_fwd(x, v, offs, k, 1e-9, 1e-6)
        assert np.allclose(S, O.exact_topk_sum(x, v, offs, k), rtol=1e-9, atol=1e-9)
        assert np.all((m < 1e-6) | (m > 1 - 1e-6))


def test_gradients_vs_finite_differences():
    x, v, offs = _case(4, sizes=(3, 9, 14))
    k, tau, tau_r = 4, 0.4, 0.7
    r0 = np.random.default_rng(5)
    dS = r0.standard_normal(len(offs) - 1)
    dm = r0.standard_normal(x.shape[0])
    dr = r0.standard_normal(x.shape[0])

    def L(xx, vv):
        r, m, S = O.soft_topk_fwd(xx, vv, offs, k, tau, tau_r)
        return float(dS @ S + dm @ m + dr @ r)

    _, m, _ = O.soft_topk_fwd(x, v, offs, k, tau, tau_r)
    dx, dv = O.soft_topk_bwd(x, v, offs, k, tau, tau_r, m, dS=dS, dm=dm, dr=dr)
    h = 1e-6
    for i in range(x.shape[0]):
        e = np.zeros_like(x)
        e[i] = h
        assert abs((L(x + e, v) - L(x - e, v)) / (2 * h) - dx[i]) <= 1e-6 * max(1.0, abs(dx[i]))
        assert abs((L(x, v + e) - L(x, v - e)) / (2 * h) - dv[i]) <= 1e-6 * max(1.0, abs(dv[i]))
