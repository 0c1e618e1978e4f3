"""Pins for the fp64 glyph-CNN oracle of the trainable query (Sec. 3
training loop; Sec. 4 softmax as a proxy for argmax; Sec. 5.5).

Checked against library routines for the special cases they cover
(scipy correlate for the convolutions, torch's bfloat16 cast for the
rounding helper) and against float64 central finite differences of the whole
query loss.
"""
import numpy as np
import pytest
import scipy.signal
import torch

import gen
from oracle import cnn


def _params(seed=5):
    return {k: v.astype(np.float64) for k, v in gen.cnn_params(seed).items()}


def _grid(n=1, seed=3):
    img, lab = gen.glyph_grids(n, seed)
    return img, lab


def test_bf16_rounding_matches_torch():
    r = np.random.default_rng(0)
    a = np.concatenate([r.standard_normal(10000) * 10.0 ** r.integers(-6, 6, 10000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(a), ref)
    assert cnn.bf16(1 + 2 ** -8) == 1.0 and cnn.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6


def test_split_cells_layout():
    img, _ = _grid(2)
    cells = cnn.split_cells(img)
    assert cells.shape == (32, 28, 28)
    assert np.array_equal(cells[16 + 4 * 2 + 3], img[1, 56:84, 84:112])


def test_conv_layers_are_scipy_correlate():
    p = _params()
    img, _ = _grid(1)
    fw = cnn.forward(p, img, quant=False)
    x0 = fw["x0"]
    for b in (0, 7):
        for co in (0, 13, 31):
            z = scipy.signal.correlate2d(x0[b], p["conv1_w"][co], mode="valid") + p["conv1_b"][co]
            assert np.allclose(fw["y1"][b, :, :, co], np.maximum(z, 0), atol=1e-12)
        for co in (0, 40, 63):
            z = scipy.signal.correlate(fw["y1"][b], p["conv2_w"][co], mode="valid")[:, :, 0] + p["conv2_b"][co]
            assert np.allclose(fw["a2"][b, :, :, co], np.maximum(z, 0), atol=1e-10)


def test_pool_takes_first_maximum():
    p = _params()
    img, _ = _grid(1)
    fw = cnn.forward(p, img, quant=False)
    a2 = fw["a2"]
    b, py, px, c = 3, 5, 7, 11
    win = [a2[b, 2 * py + dy, 2 * px + dx, c] for dy in (0, 1) for dx in (0, 1)]
    assert fw["y2"][b, py, px, c] == max(win)
    assert fw["arg"][b, py, px, c] == int(np.argmax(win))
    # all-zero windows (ReLU) pick position 0
    zero = (a2.reshape(16, 12, 2, 12, 2, 64).max(axis=(2, 4)) == 0)
    assert np.all(fw["arg"][zero] == 0)


def test_softmax_rows_sum_to_one_and_query_shape():
    p = _params()
    img, lab = _grid(2)
    fw = cnn.forward(p, img, quant=True)
    assert np.allclose(fw["P"].sum(axis=1), 1.0)
    assert fw["pred"].shape == (2, 14)
    assert np.allclose(fw["pred"][:, :10].sum(axis=1), 16.0)
    t = cnn.targets_from_labels(lab)
    assert np.array_equal(t[:, :10].sum(axis=1), [16, 16])
    assert np.array_equal(t[:, 10:], lab.sum(axis=2))


@pytest.mark.parametrize("name,idx", [
    ("fc2_b", (3,)), ("fc2_w", (2, 17)), ("fc1_b", (5,)), ("fc1_w", (9, 4000)),
    ("conv2_b", (12,)), ("conv2_w", (7, 1, 2, 30)), ("conv1_b", (4,)), ("conv1_w", (20, 0, 1)),
])
def test_whole_query_gradient_vs_finite_differences(name, idx):
    p = _params()
    img, lab = _grid(1, seed=11)
    t = cnn.targets_from_labels(lab)
    fw = cnn.forward(p, img, quant=False)
    g = cnn.backward(p, fw, t)
    h = 1e-6
    pp = {k: v.copy() for k, v in p.items()}
    pp[name][idx] += h
    lp = cnn.loss(cnn.forward(pp, img, quant=False)["pred"], t)
    pp[name][idx] -= 2 * h
    lm = cnn.loss(cnn.forward(pp, img, quant=False)["pred"], t)
    fd = (lp - lm) / (2 * h)
    scale = max(np.abs(g[name]).max(), 1e-12)
    assert abs(fd - g[name][idx]) <= 1e-5 * scale + 1e-10, (fd, g[name][idx])


def test_quantised_forward_is_close_to_fp64():
    p = _params()
    img, _ = _grid(1)
    a = cnn.forward(p, img, quant=False)["pred"]
    b = cnn.forward(p, img, quant=True)["pred"]
    assert np.allclose(a, b, rtol=2e-2, atol=2e-2)


def test_adam_first_step_closed_form():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    z = {"w": np.zeros(3)}
    newp, m, v = cnn.adam_step(p, g, z, z, t=1, lr=0.01)
    # first step: mhat = g, vhat = g^2, so the move is lr * g / (|g| + eps)
    assert np.allclose(newp["w"], p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m["w"], 0.1 * g["w"]) and np.allclose(v["w"], 0.001 * g["w"] ** 2)


def test_two_head_query_gradients_vs_finite_differences():
    """The Digit x Size query loss (float64 network, no rounding): analytic
    gradients of one element of every parameter tensor of both heads and the
    trunk against central differences."""
    import gen
    from oracle import cnn as O
    img, dig, siz = gen.glyph_grids_sized(1, 5)
    p = {k: np.asarray(v, np.float64) for k, v in gen.cnn_params(5).items()}
    q = {k: np.asarray(v, np.float64) for k, v in gen.size_head_params(5).items()}
    tgt = O.targets2(dig, siz) + 0.3  # away from the optimum: non-zero gradients
    fw = O.forward2(p, q, img, quant=False)
    g = O.backward2(p, q, fw, tgt)

    def loss(pp, qq):
        return O.loss(O.forward2(pp, qq, img, quant=False)["pred2"], tgt)

    r = np.random.default_rng(3)
    h = 1e-6
    for name in list(p) + list(q):
        src = p if name in p else q
        idx = tuple(int(r.integers(0, s)) for s in src[name].shape)
        plus = {k: v.copy() for k, v in src.items()}
        minus = {k: v.copy() for k, v in src.items()}
        plus[name][idx] += h
        minus[name][idx] -= h
        if src is p:
            fd = (loss(plus, q) - loss(minus, q)) / (2 * h)
        else:
            fd = (loss(p, plus) - loss(p, minus)) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-5 * max(1e-3, abs(g[name][idx])), name
