"""Pins of the LLP oracle (Sec. 5.3, 5.4) to brute force, invariants,
special cases and finite differences."""
import numpy as np

import gen
from oracle import llp


def test_bag_counts_brute_force_and_ragged_tail():
    r = np.random.default_rng(1)
    for n, B, K in ((1, 1, 2), (17, 4, 2), (100, 7, 3), (64, 64, 2), (65, 64, 2), (10, 512, 2)):
        y = r.integers(0, K, n)
        cnt = llp.bag_counts(y, B, K)
        assert cnt.shape == ((n + B - 1) // B, K)
        for j in range(cnt.shape[0]):
            rows = list(range(j * B, min(n, (j + 1) * B)))
            for k in range(K):
                assert cnt[j, k] == sum(1 for i in rows if y[i] == k)
            assert cnt[j].sum() == len(rows)


def test_dp_counts_scale():
    c = np.array([[3, 5], [0, 8]])
    assert np.array_equal(llp.dp_counts(c, np.zeros((2, 2)), 0.1), c)
    assert np.array_equal(llp.dp_counts(c, np.ones((2, 2)), 0.1), c + 20.0)  # 2 / 0.1
    # the mean absolute added noise is the Laplace scale 2 / eps
    z = gen.laplace_noise(20000, 2, 3)
    added = llp.dp_counts(np.zeros((20000, 2)), z, 0.1)
    assert abs(np.abs(added).mean() - 20.0) < 0.5


def test_saturated_softmax_gives_exact_counts_of_the_predictions():
    """Logits scaled up until the softmax is one-hot: the soft COUNT per bag
    equals the exact COUNT of the arg-max predictions (Sec. 4's soft
    operators reduce to the exact ones)."""
    X, _ = gen.llp_table(500, 4)
    r = np.random.default_rng(2)
    W, b = r.standard_normal((2, 6)), r.standard_normal(2)
    keep = np.abs(np.diff(X.astype(np.float64) @ W.T + b, axis=1))[:, 0] > 1e-3
    X = X[keep]
    fw = llp.forward(X, W * 1e6, b * 1e6, 16)
    exact = llp.bag_counts(llp.predict(X, W, b), 16, 2)
    assert np.array_equal(fw["cnt"], exact.astype(np.float64))


def test_forward_invariants():
    X, _ = gen.llp_table(300, 5)
    r = np.random.default_rng(3)
    W, b = r.standard_normal((3, 6)), r.standard_normal(3)
    fw = llp.forward(X, W, b, 32)
    sizes = np.bincount(np.arange(300) // 32)
    assert np.allclose(fw["cnt"].sum(axis=1), sizes, rtol=1e-12)  # each row counted once
    # bag size 1: the soft counts are the probabilities themselves
    assert np.array_equal(llp.forward(X, W, b, 1)["cnt"], fw["P"])
    # rows permuted within their bags: counts and gradients unchanged
    perm = np.concatenate([np.arange(j, min(300, j + 32))[::-1] for j in range(0, 300, 32)])
    t = fw["cnt"] + r.standard_normal(fw["cnt"].shape)
    g1 = llp.backward(X, fw, t, 32)
    fw2 = llp.forward(X[perm], W, b, 32)
    g2 = llp.backward(X[perm], fw2, t, 32)
    assert np.allclose(fw2["cnt"], fw["cnt"], rtol=1e-12)
    assert np.allclose(g1["W"], g2["W"], rtol=1e-10) and np.allclose(g1["b"], g2["b"], rtol=1e-10)
    # at the targets the gradient vanishes
    g0 = llp.backward(X, fw, fw["cnt"], 32)
    assert np.abs(g0["W"]).max() == 0.0 and np.abs(g0["b"]).max() == 0.0


def test_gradients_vs_finite_differences():
    X, y = gen.llp_table(203, 6)  # ragged last bag
    B = 16
    r = np.random.default_rng(4)
    W, b = r.standard_normal((2, 6)) * 0.5, r.standard_normal(2) * 0.5
    t = llp.bag_counts(y, B).astype(np.float64)
    fw = llp.forward(X, W, b, B)
    g = llp.backward(X, fw, t, B)

    def L(W_, b_):
        return llp.loss(llp.forward(X, W_, b_, B)["cnt"], t)

    h = 1e-6
    for i in range(2):
        for j in range(6):
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            fd = (L(Wp, b) - L(Wm, b)) / (2 * h)
            assert abs(fd - g["W"][i, j]) <= 1e-6 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (L(W, bp) - L(W, bm)) / (2 * h)
        assert abs(fd - g["b"][i]) <= 1e-6 * max(1.0, abs(fd))


def test_llp_table_shape_and_label_rate():
    X, y = gen.llp_table(50000, 7)
    assert X.shape == (50000, 6) and X.dtype == np.float32 and y.dtype == np.int32
    assert 0.2 < y.mean() < 0.28
