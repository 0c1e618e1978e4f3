"""GPU parity of the two-attribute (Digit x Size) trainable query against the
float64 oracle, and its learned-part gain test.

The query: the CNN's hidden layer feeds a digit head and a size head, and
the soft COUNT of every (digit, size) pair per grid (Sec. 4 soft group-by
over two PE attributes) is trained against the exact pair counts on true
labels.  Tolerances as in the single-attribute tests: the trunk's
tensor-core layers round to bf16 where the oracle does, so layer outputs
agree to about one bf16 ulp and whole-network gradients to 3e-2 in relative
L2 norm per tensor; the standalone pair count is plain fp32 arithmetic on
fp32 inputs (16 products per output), compared at rel 1e-6.
"""
import numpy as np
import pytest
import torch

import gen
from oracle import cnn as O
from oracle import soft
from paper_2211_02753_b300 import cnn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n", [1, 37, 1000])
def test_pe_groupby2_fwd_bwd_and_exact_count2(n):
    r = np.random.default_rng(n)
    Pa = r.random((n * 16, 10)).astype(np.float32)
    Pb = r.random((n * 16, 2)).astype(np.float32)
    cnt = cnn.pe_groupby2_fwd(dev(Pa), dev(Pb), n)
    ref = soft.pe_groupby2_fwd(Pa, Pb)
    assert np.allclose(cnt.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)
    d = r.standard_normal((n, 10, 2)).astype(np.float32)
    dPa, dPb = cnn.pe_groupby2_bwd(dev(d), dev(Pa), dev(Pb))
    ra, rb = soft.pe_groupby2_bwd(d, Pa, Pb)
    assert np.allclose(dPa.cpu().numpy(), ra, rtol=1e-5, atol=1e-5)
    assert np.allclose(dPb.cpu().numpy(), rb, rtol=1e-5, atol=1e-5)
    # one-hot PE columns: the soft pair COUNT is the exact pair COUNT bitwise
    dig = r.integers(0, 10, (n, 4, 4))
    siz = r.integers(0, 2, (n, 4, 4))
    oh = cnn.pe_groupby2_fwd(dev(np.eye(10, dtype=np.float32)[dig.reshape(-1)]),
                             dev(np.eye(2, dtype=np.float32)[siz.reshape(-1)]), n)
    assert np.array_equal(oh.cpu().numpy(), soft.exact_groupby2(dig, siz).astype(np.float32))
    # exact pair query on logits (first arg-max per attribute), with ties
    la = r.integers(-2, 3, (n * 16, 10)).astype(np.float32)
    lb = r.integers(-1, 2, (n * 16, 2)).astype(np.float32)
    ga, gb, gc = cnn.exact_count2(dev(la), dev(lb), n)
    ea, eb = np.argmax(la, axis=1), np.argmax(lb, axis=1)
    assert np.array_equal(ga.cpu().numpy(), ea) and np.array_equal(gb.cpu().numpy(), eb)
    assert np.array_equal(gc.cpu().numpy(), soft.exact_groupby2(ea.reshape(n, 4, 4), eb.reshape(n, 4, 4)))


def _pair_batch(n_grids, seed):
    img, dig, siz = gen.glyph_grids_sized(n_grids, seed)
    return img, dig, siz, O.targets2(dig, siz)


def test_pair_forward_matches_oracle():
    img, dig, siz, t = _pair_batch(3, 33)
    p, q = gen.cnn_params(5), gen.size_head_params(5)
    m = cnn.GlyphQuery2(p, q, DEV)
    b = m.forward(dev(img))
    torch.cuda.synchronize()
    fw = O.forward2(p, q, img, quant=True)
    lg = b["logits_s"].cpu().numpy()
    assert np.abs(lg - fw["logits_s"]).max() <= 2e-2 * np.abs(fw["logits_s"]).max()
    assert np.abs(b["Ps"].cpu().numpy() - fw["Ps"]).max() <= 2e-2
    pr = b["pred2"].cpu().numpy()
    assert np.abs(pr - fw["pred2"]).max() <= 2e-2
    assert np.allclose(pr.sum(axis=1), 16.0, atol=1e-4)  # every cell counted once


@pytest.mark.parametrize("n_grids", [2, 67])
def test_pair_train_step_gradients_match_oracle(n_grids):
    """67 grids: the per-grid gradient partials reduced across more grids than
    one slice of the fixed-order reduction."""
    img, dig, siz, t = _pair_batch(n_grids, 43 + n_grids)
    t = t + 0.25  # away from any optimum
    p, q = gen.cnn_params(6), gen.size_head_params(6)
    m = cnn.GlyphQuery2(p, q, DEV)
    b = m.forward(dev(img), dev(t.astype(np.float32)))
    m.backward(dev(img))
    torch.cuda.synchronize()
    fw = O.forward2(p, q, img, quant=True)
    ref = O.backward2(p, q, fw, t)
    lo = O.loss(fw["pred2"], t)
    assert abs(float(b["loss"].item()) - lo) <= 1e-3 * lo
    for k in list(cnn.PARAMS) + list(cnn.SIZE_PARAMS):
        g = m.g[k].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - ref[k]) / max(np.linalg.norm(ref[k]), 1e-30)
        assert err <= 3e-2, (k, err)


def test_pair_checkpoint_resume_bitwise():
    img, dig, siz, t = _pair_batch(4, 53)
    g_img, tg = dev(img), dev(t.astype(np.float32))
    a = cnn.GlyphQuery2(gen.cnn_params(8), gen.size_head_params(8), DEV)
    for _ in range(3):
        a.train_step(g_img, tg)
    st = a.state()
    la = a.train_step(g_img, tg)
    b = cnn.GlyphQuery2(gen.cnn_params(9), gen.size_head_params(9), DEV)
    b.load_state(st)
    lb = b.train_step(g_img, tg)
    torch.cuda.synchronize()
    assert float(la.item()) == float(lb.item())
    for k in a.p:
        assert torch.equal(a.p[k], b.p[k]), k


def pair_accuracy(cnt, dig, siz):
    """Fraction of grids whose exact pair query on predicted labels equals
    the exact pair query on the true labels (all 20 counts)."""
    e = soft.exact_groupby2(dig, siz)
    return float(np.all(cnt.reshape(len(e), -1) == e.reshape(len(e), -1), axis=1).mean())


def test_pair_query_learned_part_gain():
    """Trained only through the soft pair COUNT (no per-cell labels, no row
    sums), both heads learn the cell attributes: the exact pair query on
    held-out grids beats random init and the training-mean prior by far."""
    tr_img, tr_dig, tr_siz = gen.glyph_grids_sized(4096, gen.BASE_SEED + 6)
    te_img, te_dig, te_siz = gen.glyph_grids_sized(1024, gen.BASE_SEED + 106)
    targets = O.targets2(tr_dig, tr_siz).astype(np.float32)
    m = cnn.GlyphQuery2(gen.cnn_params(gen.BASE_SEED + 5), gen.size_head_params(gen.BASE_SEED + 5), DEV,
                        lr=1e-3, warmup=400)
    g_te = dev(te_img)
    _, _, c0 = m.exact_query(g_te)
    acc_init = pair_accuracy(c0.cpu().numpy(), te_dig, te_siz)
    g_tr, t_tr = dev(tr_img), dev(targets)
    B, steps = 256, 2400
    hist = torch.empty(steps, dtype=torch.float32, device=DEV)
    for step in range(steps):  # 150 epochs of the 4096 training grids
        i = (step % (4096 // B)) * B
        m.train_step(g_tr[i:i + B], t_tr[i:i + B], loss_out=hist[step:step + 1])
    losses = hist.cpu().tolist()
    ld, ls, c1 = m.exact_query(g_te)
    acc = pair_accuracy(c1.cpu().numpy(), te_dig, te_siz)
    dig_acc = float((ld.cpu().numpy().reshape(-1, 4, 4) == te_dig).mean())
    siz_acc = float((ls.cpu().numpy().reshape(-1, 4, 4) == te_siz).mean())
    prior = np.rint(targets.mean(axis=0)).astype(np.int64)
    acc_prior = pair_accuracy(np.tile(prior, (1024, 1)), te_dig, te_siz)
    print("pair query acc: init %.3f prior %.3f trained %.3f; digit cell acc %.4f size cell acc %.4f; "
          "loss %.3f -> %.4f" % (acc_init, acc_prior, acc, dig_acc, siz_acc, losses[0], losses[-1]))
    assert losses[-1] < 0.1 * losses[0]
    assert siz_acc >= 0.98 and dig_acc >= 0.95
    assert acc - max(acc_init, acc_prior) >= 0.5
