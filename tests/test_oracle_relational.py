"""Pins for the relational oracle (exact SQL semantics; Sec. 2 GROUP BY
COUNT, Sec. 5.2 WHERE + AVG, joins and top-k as relational operators).

The C oracle is checked against things other than itself: hand-computed
aggregates (tests/golden), an independent pure-Python brute force (nested
loops, dicts, exact rationals), numpy's stable sort as the textbook special
case of the pair sort, and conservation invariants on a full-size table.
"""
import json
import os

import numpy as np
import pytest

import gen
from oracle import brute
from oracle import relational as R

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_avg_rounding_hand_cases():
    cases = {(5, 2): 3, (-5, 2): -3, (4, 3): 1, (5, 3): 2, (-4, 3): -1, (-5, 3): -2,
             (0, 7): 0, (1, 2): 1, (-1, 2): -1, (7, 2): 4, (3, 2): 2, (-3, 2): -2, (201, 2): 101}
    for (s, c), q in cases.items():
        assert R.avg_round(s, c) == q, (s, c)
        assert brute.avg_half_away(s, c) == q, (s, c)


def test_groupby_hand_computed_8_rows():
    g = _load("groupby_8rows.json")
    c = {k: np.array(v, dtype=np.int64) for k, v in g["columns"].items()}
    cols = {"flag": c["flag"].astype(np.int8), "status": c["status"].astype(np.int8),
            "qty": c["qty"], "price": c["price"], "disc": c["disc"], "date": c["date"].astype(np.int32)}
    sel = R.filter([(cols["date"], "<=", 2460)], 8)
    assert sel.tolist() == g["filter_rows"]
    keys, aggs = R.groupby([cols["flag"], cols["status"]],
                           [("count", None, None, None), ("sum", cols["qty"], None, None),
                            ("sum", cols["price"], None, None),
                            ("sum_mul_kminus", cols["price"], cols["disc"], 100),
                            ("avg", cols["qty"], None, None)], 8, sel=sel)
    assert keys.tolist() == [gr["key"] for gr in g["groups"]]
    exp = [[gr["count"], gr["sum_qty"], gr["sum_price"], gr["sum_disc_price"], gr["avg_qty"]] for gr in g["groups"]]
    assert aggs.tolist() == exp


def test_avg_ties_fixture():
    g = _load("groupby_8rows.json")["avg_ties"]
    k = np.array(g["k"], np.int32)
    v = np.array(g["v"], np.int64)
    keys, aggs = R.groupby([k], [("avg", v, None, None)], len(k))
    assert {str(a): b for a, b in zip(keys[:, 0].tolist(), aggs[:, 0].tolist())} == g["avg"]


def _tiny_table(seed, n):
    r = np.random.default_rng(seed)
    return {
        "k1": r.integers(-3, 4, n).astype(np.int8),
        "k2": r.integers(0, 5, n).astype(np.int32),
        "a": r.integers(-10**9, 10**9, n).astype(np.int64),
        "b": r.integers(0, 11, n).astype(np.int64),
        "d": r.integers(0, 100, n).astype(np.int32),
    }


@pytest.mark.parametrize("seed", range(12))
def test_filter_and_groupby_vs_brute(seed):
    n = [0, 1, 2, 7, 64, 300][seed % 6] + seed
    t = _tiny_table(seed, n)
    preds = [(t["d"], ["<", "<=", ">", ">=", "==", "!="][seed % 6], 50), (t["k2"], "!=", seed % 5)]
    sel = R.filter(preds, n)
    assert sel.tolist() == brute.filter(preds, n)
    aggs = [("count", None, None, None), ("sum", t["a"], None, None),
            ("sum_mul_kminus", t["a"], t["b"], 100), ("avg", t["a"], None, None),
            ("min", t["a"], None, None), ("max", t["a"], None, None)]
    keys, vals = R.groupby([t["k1"], t["k2"]], aggs, n, sel=sel)
    ref = brute.groupby([t["k1"], t["k2"]], aggs, sel.tolist())
    assert [tuple(r) for r in keys.tolist()] == [k for k, _ in ref]
    assert [tuple(r) for r in vals.tolist()] == [v for _, v in ref]


@pytest.mark.parametrize("seed", range(10))
def test_join_vs_nested_loop(seed):
    r = np.random.default_rng(100 + seed)
    nb = [0, 1, 5, 40, 200][seed % 5]
    npr = [0, 3, 50, 300][seed % 4]
    unique = seed % 2 == 0
    bkey = (r.permutation(nb) * 3 + 1 if unique else r.integers(0, 20, nb)).astype(np.int32)
    pkey = r.integers(-2, max(3, 3 * nb + 2), npr).astype(np.int32)
    bsel = np.sort(r.choice(nb, size=nb // 2, replace=False)).astype(np.int32) if nb and seed % 3 == 0 else None
    psel = np.sort(r.choice(npr, size=npr // 2, replace=False)).astype(np.int32) if npr and seed % 4 == 1 else None
    op, ob, dup = R.join(bkey, pkey, bsel=bsel, psel=psel)
    brows = bsel.tolist() if bsel is not None else list(range(nb))
    prows = psel.tolist() if psel is not None else list(range(npr))
    ref = brute.join(bkey, brows, pkey, prows)
    assert list(zip(op.tolist(), ob.tolist())) == ref
    keys_b = bkey[brows] if len(brows) else np.zeros(0, np.int32)
    assert dup == (len(np.unique(keys_b)) != len(keys_b))


def test_join_capacity_reports_true_count():
    bkey = np.arange(10, dtype=np.int32)
    pkey = np.tile(np.arange(10, dtype=np.int32), 3)
    op, ob, _ = R.join(bkey, pkey, cap=7)
    assert len(op) == 7 and op.tolist() == list(range(7))


@pytest.mark.parametrize("seed", range(6))
def test_topk_vs_sorted(seed):
    r = np.random.default_rng(seed)
    n = [0, 1, 5, 50, 500, 2000][seed]
    vals = r.integers(-5, 6, n).astype(np.int64)  # many ties
    keys = r.permutation(n).astype(np.int64)
    for k in (1, 3, 10):
        ov, ok = R.topk(vals, keys, k)
        ref = brute.topk(vals, keys, k)
        assert list(zip(ov.tolist(), ok.tolist())) == ref


@pytest.mark.parametrize("n", [0, 1, 1000, 100000])
def test_sort_pairs_is_numpy_stable_sort(n):
    r = np.random.default_rng(n)
    keys = r.integers(0, 1 << 12, n).astype(np.uint64)  # many equal keys
    vals = np.arange(n, dtype=np.uint32)
    ok, ov = R.sort_pairs(keys, vals)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(ok, keys[order])
    assert np.array_equal(ov, vals[order])


def test_invariants_60k_fact_table():
    """Row-count and sum conservation on the 60,000-row pricing-summary table."""
    n = 60000
    t = gen.fact_table(n, 15000, gen.BASE_SEED + 0)
    sel = R.filter([(t["date"], "<=", 2460)], n)
    rej = R.filter([(t["date"], ">", 2460)], n)
    assert len(sel) + len(rej) == n
    assert len(np.intersect1d(sel, rej)) == 0
    keys, aggs = R.groupby([t["flag"], t["status"]],
                           [("count", None, None, None), ("sum", t["qty"], None, None),
                            ("sum_mul_kminus", t["price"], t["disc"], 100)], n, sel=sel)
    assert keys.tolist() == [[f, s] for f in range(3) for s in range(2)]
    assert aggs[:, 0].sum() == len(sel)
    assert aggs[:, 1].sum() == int(t["qty"][sel].sum())
    assert aggs[:, 2].sum() == int((t["price"][sel] * (100 - t["disc"][sel])).sum())
    # ~96.25% selectivity of date <= 2460 over U[0, 2556]
    assert abs(len(sel) / n - 2461 / 2557) < 0.01


def test_mutation_in_oracle_is_caught():
    """A planted mistake (a dropped row) must break the pins above: the
    brute force disagrees with a filter that loses its last row."""
    t = _tiny_table(3, 50)
    preds = [(t["d"], ">=", 0)]
    good = R.filter(preds, 50).tolist()
    assert good == brute.filter(preds, 50)
    assert good[:-1] != brute.filter(preds, 50)


def test_parallel_oracle_equals_single_thread():
    """The OpenMP row-partitioned filter, join and group-by (used to time the
    CPU baseline) give exactly the single-threaded oracle's results: row order,
    group order, every aggregate including AVG rounding, N:M join order."""
    from oracle import relational as R
    r = np.random.default_rng(77)
    n = 50_003
    a = r.integers(-5, 6, n).astype(np.int8)
    b = r.integers(0, 300, n).astype(np.int32)
    v = r.integers(-10**9, 10**9, n).astype(np.int64)
    w = r.integers(0, 11, n).astype(np.int64)
    preds = [(a, "!=", 0), (b, "<", 250)]
    sel = R.filter(preds, n)
    assert np.array_equal(R.filter(preds, n, parallel=True), sel)
    aggs = [("count", None, None, None), ("sum", v, None, None), ("sum_mul_kminus", v, w, 100), ("avg", v, None, None),
            ("min", v, None, None), ("max", b, None, None)]
    k1, a1 = R.groupby([a, b], aggs, n, sel=sel)
    k2, a2 = R.groupby([a, b], aggs, n, sel=sel, parallel=True)
    assert np.array_equal(k1, k2) and np.array_equal(a1, a2)
    k1, a1 = R.groupby([a], aggs, n)
    k2, a2 = R.groupby([a], aggs, n, parallel=True)
    assert np.array_equal(k1, k2) and np.array_equal(a1, a2)
    bk = r.integers(0, 2000, 3000).astype(np.int32)  # duplicate build keys: N:M
    pk = r.integers(0, 2200, 20001).astype(np.int32)
    p1, b1, d1 = R.join(bk, pk)
    p2, b2, d2 = R.join(bk, pk, parallel=True)
    assert d1 and d2 and np.array_equal(p1, p2) and np.array_equal(b1, b2)
    assert R.threads() >= 1
