"""GPU parity of learning from label proportions (Sec. 5.3) and its label-DP
counts (Sec. 5.4) against the float64 oracle.

Tolerances.  Bag counts of labels are integers: bit-exact.  The Laplace
counts are one fp32 multiply-add of exact inputs: rel 1e-6.  The step
kernel sums fp32 probabilities per bag (at most a few thousand terms of
[0, 1]) and fp32 per-block gradient partials added in float64: soft counts
agree to rel 1e-5, the loss to rel 1e-5, gradients to 1e-4 of their norm
(the terms cancel, so the bound is relative to the gradient's size, not
per element).  Predictions are an arg-max of fp32 logits: rows whose two
logits lie within 1e-4 of each other may go either way and are checked to
be valid; all others must match.
"""
import numpy as np
import pytest
import torch

import gen
from oracle import cnn as O
from oracle import llp as R
from paper_2211_02753_b300 import llp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n,B,K", [(1, 1, 2), (1000, 1, 2), (1003, 8, 2), (100_003, 64, 3), (5000, 512, 2),
                                   (70, 512, 4), (300_000, 4096, 2)])
def test_counts_exact_and_laplace(n, B, K):
    r = np.random.default_rng(n + B)
    y = r.integers(0, K, n).astype(np.int32)
    got = llp.counts(dev(y), B, K)
    assert np.array_equal(got.cpu().numpy(), R.bag_counts(y, B, K).astype(np.float32))
    z = gen.laplace_noise(R.n_bags(n, B), K, 5)
    got = llp.counts(dev(y), B, K, noise=dev(z), eps=0.1)
    ref = R.dp_counts(R.bag_counts(y, B, K), z, 0.1)
    assert np.allclose(got.cpu().numpy(), ref, rtol=1e-6, atol=1e-5)


def test_counts_label_out_of_range_sets_overflow_and_is_dropped():
    y = np.array([0, 1, 5, 1, -1, 0], np.int32)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = llp.counts(dev(y), 3, 2, status=st)
    assert int(st.item()) == 32
    assert got.cpu().numpy().tolist() == [[1.0, 1.0], [1.0, 1.0]]
    # bags of a warp's rows and more (the warp-per-bag kernel)
    y = np.zeros(70, np.int32)
    y[33] = 7
    y[40:50] = 1
    st.zero_()
    got = llp.counts(dev(y), 32, 2, status=st)
    assert int(st.item()) == 32
    assert got.cpu().numpy().tolist() == [[32.0, 0.0], [21.0, 10.0], [6.0, 0.0]]


CASES = [
    (1, 6, 2, 1),            # one row
    (10_007, 6, 2, 1),       # bag size 1: a thread per bag
    (10_007, 6, 2, 7),       # small bags, ragged tail
    (100_003, 6, 2, 64),     # a warp per bag
    (50_000, 6, 2, 1000),    # one bag per group
    (50_000, 6, 2, 1024),    # one bag per chunk exactly
    (20_000, 6, 2, 3000),    # bags longer than a chunk: two passes
    (500, 6, 2, 4096),       # one short bag
    (30_011, 13, 3, 32),     # the general kernel (K <= 4, d <= 16)
    (30_011, 16, 4, 2500),
    (9_999, 1, 2, 16),       # one feature
    (10_001, 1, 2, 7),       # groups of 1022 rows x 4 bytes: not whole 16-byte copies, the unpipelined kernel
    (4_321, 5, 2, 48),       # odd width, bags neither a multiple nor a divisor of 32: the unpipelined kernel
    (4_321, 5, 2, 32),       # odd width streamed: scalar feature loads, ragged copies
    (12_345, 6, 2, 2),       # bags of two lanes
    (100_003, 6, 2, 512),    # one bag per task
    (70_001, 8, 2, 256),     # the widest streamed row
    (3_000, 6, 2, 96),       # tasks of 480 rows: stages of 128, 128, 128, 96
]


def _problem(n, d, K, B, seed):
    r = np.random.default_rng(seed)
    if d == 6 and K == 2:
        X, y = gen.llp_table(n, seed)
    else:
        X = r.standard_normal((n, d)).astype(np.float32)
        y = r.integers(0, K, n).astype(np.int32)
    W = (r.standard_normal((K, d)) * 0.5).astype(np.float32)
    b = (r.standard_normal(K) * 0.5).astype(np.float32)
    t = R.bag_counts(y, B, K).astype(np.float32)
    return X, y, W, b, t


@pytest.mark.parametrize("n,d,K,B", CASES)
def test_step_matches_oracle(n, d, K, B):
    X, y, W, b, t = _problem(n, d, K, B, n + d + B)
    tr = llp.LLPTrainer(dev(X), dev(t), B, W, b)
    loss = float(tr.forward_backward(cnt_out=True).item())
    fw = R.forward(X, W, b, B)
    g = R.backward(X, fw, t, B)
    lo = R.loss(fw["cnt"], t)
    assert np.allclose(tr.cnt.cpu().numpy(), fw["cnt"], rtol=1e-5, atol=1e-5)
    assert abs(loss - lo) <= 1e-5 * lo + 1e-7
    for got, ref in ((tr.dW, g["W"]), (tr.db, g["b"])):
        got = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-9
    assert int(tr.status.item()) == 0


def test_step_misaligned_rows_take_the_plain_kernel():
    """X 4 bytes past a 16-byte boundary: no bulk copies; same results."""
    n, d, K, B = 50_003, 6, 2, 64
    X, y, W, b, t = _problem(n, d, K, B, 77)
    flat = torch.zeros(n * d + 1, dtype=torch.float32, device=DEV)
    flat[1:] = dev(X.reshape(-1))
    Xm = flat[1:].view(n, d)
    assert Xm.data_ptr() % 16 == 4
    tr = llp.LLPTrainer(Xm, dev(t), B, W, b)
    tr.forward_backward(cnt_out=True)
    fw = R.forward(X, W, b, B)
    g = R.backward(X, fw, t, B)
    assert np.allclose(tr.cnt.cpu().numpy(), fw["cnt"], rtol=1e-5, atol=1e-5)
    assert np.linalg.norm(tr.dW.cpu().numpy() - g["W"]) <= 1e-4 * np.linalg.norm(g["W"])
    assert int(tr.status.item()) == 0


def test_step_is_deterministic():
    X, y, W, b, t = _problem(200_000, 6, 2, 64, 9)
    tr = llp.LLPTrainer(dev(X), dev(t), 64, W, b)
    tr.forward_backward()
    a = (tr.loss.clone(), tr.dW.clone(), tr.db.clone())
    tr.forward_backward()
    assert torch.equal(a[0], tr.loss) and torch.equal(a[1], tr.dW) and torch.equal(a[2], tr.db)


def test_step_full_size_matches_oracle():
    """The benchmark's size (64M rows x 6 features, bags of 64, label-DP
    counts): loss and gradients against the oracle run over consecutive
    slices of whole bags (the loss and the gradients are sums over bags),
    and the soft counts of sampled bags."""
    n, B = 64_000_000, 64
    X, y = gen.llp_table(n, gen.BASE_SEED + 9)
    nb = R.n_bags(n, B)
    t = R.dp_counts(R.bag_counts(y, B), gen.laplace_noise(nb, 2, gen.BASE_SEED + 10), 0.1).astype(np.float32)
    r = np.random.default_rng(1)
    W = (r.standard_normal((2, 6)) * 0.5).astype(np.float32)
    b = np.array([0.3, -0.2], np.float32)
    tr = llp.LLPTrainer(dev(X), dev(t), B, W, b)
    loss = float(tr.forward_backward(cnt_out=True).item())
    cnt = tr.cnt.cpu().numpy()
    gW, gb = tr.dW.cpu().numpy().astype(np.float64), tr.db.cpu().numpy().astype(np.float64)
    del tr
    torch.cuda.empty_cache()
    sq, rW, rb = 0.0, np.zeros((2, 6)), np.zeros(2)
    step = 64 * 65536
    for s in range(0, n, step):
        fw = R.forward(X[s:s + step], W, b, B)
        tt = t[s // B:(s + step) // B]
        d = fw["cnt"] - tt
        sq += float((d * d).sum())
        # the slice's share of the full mean's gradient
        g = R.backward(X[s:s + step], fw, tt, B)
        scale = fw["cnt"].size / (nb * 2)
        rW += g["W"] * scale
        rb += g["b"] * scale
        if s == 0:
            assert np.allclose(cnt[:1000], fw["cnt"][:1000], rtol=1e-5, atol=1e-5)
    assert abs(loss - sq / (nb * 2)) <= 1e-5 * sq / (nb * 2)
    assert np.linalg.norm(gW - rW) <= 1e-4 * np.linalg.norm(rW)
    assert np.linalg.norm(gb - rb) <= 1e-4 * np.linalg.norm(rb)
    for j in r.integers(0, nb, 200):
        ref = R.forward(X[j * B:(j + 1) * B], W, b, B)["cnt"][0]
        assert np.allclose(cnt[j], ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("d,K", [(6, 2), (13, 3)])
def test_predict_and_error_count(d, K):
    n = 100_001
    r = np.random.default_rng(d)
    X = r.standard_normal((n, d)).astype(np.float32)
    W = r.standard_normal((K, d)).astype(np.float32)
    b = r.standard_normal(K).astype(np.float32)
    ref = r.integers(0, K, n).astype(np.int32)
    lab, err = llp.predict(dev(X), dev(W), dev(b), dev(ref))
    lab = lab.cpu().numpy()
    logits = X.astype(np.float64) @ W.T.astype(np.float64) + b
    srt = np.sort(logits, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-4
    assert np.array_equal(lab[clear], np.argmax(logits, axis=1)[clear])
    amb = ~clear  # near-ties: the GPU's choice must attain the maximum within the bound
    assert np.all(logits[amb, lab[amb]] >= srt[amb, -1] - 1e-4)
    assert int(err.item()) == int((lab != ref).sum())


def _oracle_train(X, t, B, steps, lr):
    p = {"W": np.zeros((2, 6)), "b": np.zeros(2)}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    for s in range(1, steps + 1):
        fw = R.forward(X, p["W"], p["b"], B)
        p, m, v = O.adam_step(p, R.backward(X, fw, t, B), m, v, s, lr=lr)
    return p


@pytest.mark.parametrize("B,dp", [(1, False), (64, False), (512, False), (64, True)])
def test_training_matches_oracle_training(B, dp):
    """Census-sized LLP (32,561 training rows, 16,281 test rows): 300 Adam
    steps of full-batch training on the GPU reach the oracle's parameters
    (same steps in float64) and the same test error, without and with the
    Laplace counts."""
    Xtr, ytr = gen.llp_table(32561, gen.BASE_SEED + 7)
    Xte, yte = gen.llp_table(16281, gen.BASE_SEED + 107)
    t = R.bag_counts(ytr, B).astype(np.float64)
    if dp:
        t = R.dp_counts(t, gen.laplace_noise(t.shape[0], 2, gen.BASE_SEED + 8), 0.1)
    t = t.astype(np.float32)
    steps, lr = 300, 0.05
    tr = llp.LLPTrainer(dev(Xtr), dev(t), B, np.zeros((2, 6)), np.zeros(2), lr=lr)
    for _ in range(steps):
        tr.step()
    p = _oracle_train(Xtr, t, B, steps, lr)
    W, b = tr.W.cpu().numpy().astype(np.float64), tr.b.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(W - p["W"]) <= 2e-3 * np.linalg.norm(p["W"])
    assert np.linalg.norm(b - p["b"]) <= 2e-3 * max(np.linalg.norm(p["b"]), 1e-3)
    _, err = llp.predict(dev(Xte), tr.W, tr.b, dev(yte))
    e_gpu = int(err.item()) / len(yte)
    e_ref = R.error_rate(Xte, p["W"], p["b"], yte)
    print("B=%d dp=%s: test error GPU %.4f oracle %.4f" % (B, dp, e_gpu, e_ref))
    assert abs(e_gpu - e_ref) <= 2e-3
    if not dp:
        assert e_gpu < 0.22  # well below the majority-class error (about 0.235)
