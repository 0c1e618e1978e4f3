"""fp64 oracle for learning from label proportions (Sec. 5.3) and its
label-differential-privacy variant (Sec. 5.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The query of Sec. 5.3: a linear table-valued function scores every row
(logits = x W^T + b), softmax stands in for the argmax that would pick the
class (Sec. 4), and SELECT class, COUNT(*) ... GROUP BY class runs softly on
each bag, so the bag's soft count of class k is the sum of its rows'
probabilities of k.  Training only sees the bags' count labels: the loss is
the mean squared error between the soft counts and those labels (the
trainable query's loss), minimised by Adam.  Test error is measured per row
on the hard classifier (argmax of the logits).

  bag j             rows j*B .. min(n, (j+1)*B) - 1   (the last bag may be short)
  P[i, k]           softmax_k(x_i W^T + b)
  cnt[j, k]         sum_{i in bag j} P[i, k]
  loss              mean over j, k of (cnt[j, k] - t[j, k])^2
  dcnt[j, k]        2 (cnt[j, k] - t[j, k]) / (n_bags K)
  dlogit[i, k]      P[i, k] (dcnt[j(i), k] - sum_l P[i, l] dcnt[j(i), l])
  dW = dlogit^T X,  db = sum_i dlogit[i]

Label DP (Sec. 5.4, the Laplace mechanism on the count labels): every
released count gets independent Laplace noise of scale sensitivity / eps.
Reading: the count vector of a bag moves by 1 in two classes when one row's
label changes, so its L1 sensitivity is 2, and the scale is 2 / eps
(eps = 0.1 in the paper: scale 20).  The standard Laplace draws are inputs
(``gen.laplace_noise``); this module scales and adds them.

Library primitives used as steps: numpy.exp, numpy.add.at (an indexed sum),
matrix products.
"""
from __future__ import annotations

import numpy as np

DP_SENSITIVITY = 2.0


def n_bags(n: int, B: int) -> int:
    return (n + B - 1) // B


def bag_of(n: int, B: int) -> np.ndarray:
    return np.arange(n) // B


def bag_counts(labels, B: int, K: int = 2) -> np.ndarray:
    """Exact COUNT per (bag, class) of integer labels: int64 [n_bags, K]."""
    y = np.asarray(labels).astype(np.int64)
    n = y.shape[0]
    cnt = np.zeros((n_bags(n, B), K), np.int64)
    np.add.at(cnt, (bag_of(n, B), y), 1)
    return cnt


def dp_counts(counts, noise, eps: float, sensitivity: float = DP_SENSITIVITY) -> np.ndarray:
    """The Laplace mechanism: counts + (sensitivity / eps) * noise, with
    noise the standard Laplace draws of the same shape."""
    return np.asarray(counts, np.float64) + (sensitivity / eps) * np.asarray(noise, np.float64)


def softmax(z):
    z = np.asarray(z, np.float64)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def forward(X, W, b, B: int) -> dict:
    X = np.asarray(X, np.float64)
    logits = X @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
    P = softmax(logits)
    cnt = np.zeros((n_bags(X.shape[0], B), P.shape[1]))
    np.add.at(cnt, bag_of(X.shape[0], B), P)
    return {"logits": logits, "P": P, "cnt": cnt}


def loss(cnt, target) -> float:
    d = np.asarray(cnt, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d))


def backward(X, fw: dict, target, B: int) -> dict:
    X = np.asarray(X, np.float64)
    cnt, P = fw["cnt"], fw["P"]
    dcnt = 2.0 * (cnt - np.asarray(target, np.float64)) / cnt.size
    dP = dcnt[bag_of(X.shape[0], B)]
    dlogit = P * (dP - (P * dP).sum(axis=1, keepdims=True))
    return {"W": dlogit.T @ X, "b": dlogit.sum(axis=0)}


def predict(X, W, b) -> np.ndarray:
    """Hard classifier: first arg-max of the logits."""
    X = np.asarray(X, np.float64)
    return np.argmax(X @ np.asarray(W, np.float64).T + np.asarray(b, np.float64), axis=1)


def error_rate(X, W, b, labels) -> float:
    return float(np.mean(predict(X, W, b) != np.asarray(labels)))
