"""GPU parity of the relational operators against the CPU oracle: bit-exact
(row ids, keys, int64 aggregates, order).  Inputs are seeded (gen) and the
expected values come from oracle/ only."""
import numpy as np
import pytest
import torch

import gen
from oracle import relational as R
from paper_2211_02753_b300 import ops
from paper_2211_02753_b300._lib import TdpError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def np_(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def _table(n, seed):
    r = np.random.default_rng(seed)
    return {
        "a8": r.integers(-128, 128, n).astype(np.int8),
        "u8": r.integers(0, 256, n).astype(np.uint8),
        "b32": r.integers(-1000, 1000, n).astype(np.int32),
        "c64": r.integers(-10**12, 10**12, n).astype(np.int64),
        "k1": r.integers(0, 3, n).astype(np.int8),
        "k2": r.integers(-2, 3, n).astype(np.int32),
        "v": r.integers(-10**9, 10**9, n).astype(np.int64),
        "w": r.integers(0, 11, n).astype(np.int64),
    }


SIZES = [0, 1, 3, 4095, 4096, 4097, 70001]


@pytest.mark.parametrize("n", SIZES)
def test_filter_matches_oracle(n):
    t = _table(n, n)
    names = ["a8", "u8", "b32", "c64"]
    cols = [cu(t[k]) for k in names]
    preds = [(0, ">", -60), (1, "!=", 7), (2, "<=", 500), (3, ">=", -5 * 10**11)]
    out = ops.filter(cols, preds, gather=[0, 3])
    ops.check(out["status"])
    ref = R.filter([(t[names[c]], op, lit) for c, op, lit in preds], n)
    cnt = int(out["count"].item())
    assert cnt == len(ref)
    assert np.array_equal(np_(out["rowid"], cnt), ref)
    assert np.array_equal(np_(out["gathered"][0], cnt), t["a8"][ref])
    assert np.array_equal(np_(out["gathered"][1], cnt), t["c64"][ref])


@pytest.mark.parametrize("op", ["<", "<=", ">", ">=", "==", "!="])
def test_filter_each_comparison_and_no_predicate(op):
    n = 20000
    t = _table(n, 7)
    cols = [cu(t["b32"])]
    out = ops.filter(cols, [(0, op, 3)])
    ref = R.filter([(t["b32"], op, 3)], n)
    assert np.array_equal(np_(out["rowid"], int(out["count"].item())), ref)
    out = ops.filter(cols, [])
    assert int(out["count"].item()) == n


def test_filter_unaligned_columns_and_capacity():
    n = 10001
    t = _table(n + 1, 3)
    base = cu(t["b32"])
    col = base[1:]  # 4-byte offset: the scalar load path
    assert col.data_ptr() % 16 != 0
    ref = R.filter([(t["b32"][1:], "<", 0)], n)
    out = ops.filter([col], [(0, "<", 0)])
    assert np.array_equal(np_(out["rowid"], int(out["count"].item())), ref)
    cap = len(ref) // 2
    out = ops.filter([col], [(0, "<", 0)], capacity=cap)
    assert int(out["count"].item()) == len(ref)
    assert int(out["status"].item()) & 4
    assert np.array_equal(np_(out["rowid"], cap), ref[:cap])


@pytest.mark.parametrize("n", [16384, 50000])
def test_filter_literals_outside_the_column_type(n):
    """Range form of each comparison at and beyond the bounds of int8, uint8
    and int32 columns (literals that clamp, or make the test empty or total),
    over several full tiles and a ragged one."""
    t = _table(n, 11)
    names = ["a8", "u8", "b32"]
    cols = [cu(t[k]) for k in names]
    big = 2**40
    cases = [(0, "<", 200), (0, ">", 200), (0, "==", 300), (0, "!=", 300), (0, ">=", -200), (0, "<=", -129),
             (0, "<", -128), (0, ">", 127), (0, ">=", 127), (0, "<=", -128),
             (1, "<", 0), (1, ">=", 0), (1, "<=", 255), (1, ">", 255), (1, "==", -1), (1, "!=", 256),
             (2, "<", -big), (2, ">", -big), (2, "<=", big), (2, ">=", big), (2, "<", -(2**63)),
             (2, ">", 2**63 - 1), (2, "==", 999), (2, "!=", -1000)]
    for c, op, lit in cases:
        out = ops.filter(cols, [(c, op, lit)], gather=[2])
        ops.check(out["status"])
        ref = R.filter([(t[names[c]], op, lit)], n)
        cnt = int(out["count"].item())
        assert cnt == len(ref), (c, op, lit)
        assert np.array_equal(np_(out["rowid"], cnt), ref), (c, op, lit)
        assert np.array_equal(np_(out["gathered"][0], cnt), t["b32"][ref]), (c, op, lit)


def test_filter_device_row_count():
    """The row count read on the device (d_n) cuts the table inside a tile."""
    n = 70000
    t = _table(n, 12)
    cols = [cu(t["u8"])]
    for m in (0, 1, 16383, 16385, 69999):
        d_n = torch.tensor([m], dtype=torch.int64, device=DEV)
        out = ops.filter(cols, [(0, ">=", 100)], gather=[0], d_n=d_n)
        ops.check(out["status"])
        ref = R.filter([(t["u8"][:m], ">=", 100)], m)
        cnt = int(out["count"].item())
        assert cnt == len(ref)
        assert np.array_equal(np_(out["rowid"], cnt), ref)
        assert np.array_equal(np_(out["gathered"][0], cnt), t["u8"][ref])


def test_filter_multi_round():
    """100M one-byte rows are more than one round of chunks (every block's
    chunk is capped by its shared-memory bitmap), so the table is counted and
    written in two rounds; row ids alone take the bulk-store write path, a
    gathered column the per-lane path."""
    n = 100_000_000
    u = np.random.default_rng(7).integers(0, 256, n).astype(np.uint8)
    g = cu(u)
    ref = R.filter([(u, ">=", 128)], n)
    out = ops.filter([g], [(0, ">=", 128)])
    ops.check(out["status"])
    cnt = int(out["count"].item())
    assert cnt == len(ref)
    assert np.array_equal(np_(out["rowid"], cnt), ref)
    del out
    out = ops.filter([g], [(0, ">=", 128)], gather=[0])
    ops.check(out["status"])
    assert int(out["count"].item()) == len(ref)
    assert np.array_equal(np_(out["rowid"], cnt), ref)
    assert np.array_equal(np_(out["gathered"][0], cnt), u[ref])


def test_filter_config1_60m_rows():
    n = 60_000_000
    t = gen.fact_table(n, 15_000_000, gen.BASE_SEED + 1, cols=("date",))
    out = ops.filter([cu(t["date"])], [(0, "<=", 2460)])
    ops.check(out["status"])
    ref = R.filter([(t["date"], "<=", 2460)], n)
    cnt = int(out["count"].item())
    assert cnt == len(ref)
    got = np_(out["rowid"], cnt)
    assert np.array_equal(got, ref)


AGGS6 = [("count", None, None, None), ("sum", 6, None, None), ("sum_mul_kminus", 6, 7, 100),
         ("avg", 6, None, None), ("min", 6, None, None), ("max", 6, None, None)]


def _oracle_aggs(t, names):
    out = []
    for op, a, b, k in AGGS6:
        out.append((op, t[names[a]] if a is not None else None, t[names[b]] if b is not None else None, k))
    return out


@pytest.mark.parametrize("strategy", ["small_domain", "sort", "partition"])
@pytest.mark.parametrize("n", [0, 1, 4097, 70001])
def test_groupby_matches_oracle(strategy, n):
    t = _table(n, 100 + n)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    cols = [cu(t[k]) for k in names]
    cols[4] = ops.Col(cols[4], 0, 2)
    cols[5] = ops.Col(cols[5], -2, 2)
    preds = [(2, "<", 700)]
    out = ops.groupby_agg(cols, [4, 5], AGGS6, preds=preds, strategy=strategy)
    ops.check(out["status"])
    sel = R.filter([(t["b32"], "<", 700)], n)
    rk, ra = R.groupby([t["k1"], t["k2"]], _oracle_aggs(t, names), n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["keys"][1], g), rk[:, 1])
    for j in range(len(AGGS6)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), AGGS6[j]


# Private per-thread tables (at most 63 accumulators) over millions of rows,
# with ragged tails, a device row count and an unaligned column.
STREAM_CASES = [
    ([4], [("count", None, None, None), ("sum", 6, None, None), ("sum_mul_kminus", 6, 7, 100),
           ("min", 0, None, None), ("max", 3, None, None), ("avg", 2, None, None)]),
    ([4, 5], [("count", None, None, None), ("sum", 6, None, None), ("avg", 7, None, None)]),
    # four slots with MIN / MAX beside one a * (k - b) slot (not purely additive)
    ([4], [("min", 0, None, None), ("sum_mul_kminus", 6, 7, 100), ("max", 3, None, None),
           ("count", None, None, None)]),
]


@pytest.mark.parametrize("n", [1_048_576, 1_048_579, 5_000_001])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_groupby_small_domain_streamed(n, case):
    keys, aggs = STREAM_CASES[case]
    t = _table(n, 900 + n + case)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    cols = [cu(t[k]) for k in names]
    cols[4] = ops.Col(cols[4], 0, 2)
    cols[5] = ops.Col(cols[5], -2, 2)
    preds = [(2, "<", 700), (1, ">=", 10)]
    out = ops.groupby_agg(cols, keys, aggs, preds=preds, strategy="small_domain")
    ops.check(out["status"])
    sel = R.filter([(t["b32"], "<", 700), (t["u8"], ">=", 10)], n)
    oa = [(op, t[names[a]] if a is not None else None, t[names[b]] if b is not None else None, kk)
          for op, a, b, kk in aggs]
    rk, ra = R.groupby([t[names[k]] for k in keys], oa, n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    for j in range(len(keys)):
        assert np.array_equal(np_(out["keys"][j], g), rk[:, j])
    for j in range(len(aggs)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), aggs[j]


def test_groupby_small_domain_streamed_device_count_and_unaligned_column():
    n, m = 3_000_000, 2_000_123
    keys, aggs = STREAM_CASES[0]
    t = _table(n, 77)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    oa = [(op, t[names[a]] if a is not None else None, t[names[b]] if b is not None else None, kk)
          for op, a, b, kk in aggs]
    sel = R.filter([(t["b32"][:m], "<", 700)], m)
    rk, ra = R.groupby([t["k1"][:m]], oa, m, sel=sel)
    for unaligned in (False, True):
        cols = [cu(t[k]) for k in names]
        if unaligned:  # a 4-byte offset: scalar loads instead of vector loads
            buf = torch.zeros(n + 1, dtype=torch.int32, device=DEV)
            buf[1:] = cols[2]
            cols[2] = buf[1:]
            assert cols[2].data_ptr() % 16 == 4
        cols[4] = ops.Col(cols[4], 0, 2)
        nsel = torch.tensor([m], dtype=torch.int64, device=DEV)
        out = ops.groupby_agg(cols, keys, aggs, preds=[(2, "<", 700)], n=n, nsel=nsel, strategy="small_domain")
        ops.check(out["status"])
        g = int(out["ngroups"].item())
        assert g == len(rk)
        assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
        for j in range(len(aggs)):
            assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), (unaligned, aggs[j])


# Additive aggregates over small tables (at most 45 accumulators: 32 groups x
# 1 slot, 15 x 2, 6 x 5, 15 x 3 with the product slot first) on the
# small-domain strategy: keys k1 (3 values) x
# k2 (5), a8 & 31 as a bounded column of 32 groups, u8 % 6 as 6 groups.
ADD_CASES = [
    ("a32", [("count", None, None, None)]),                                          # 32 groups x 1 slot
    ("k12", [("count", None, None, None), ("sum", 6, None, None)]),                   # 15 x 2
    ("g6", [("sum", 6, None, None), ("sum", 3, None, None), ("sum_mul_kminus", 6, 7, 100),
            ("count", None, None, None), ("avg", 2, None, None)]),                  # 6 x 5
    ("k12", [("sum_mul_kminus", 6, 7, 100), ("count", None, None, None), ("sum", 3, None, None)]),  # 15 x 3
]


@pytest.mark.parametrize("n", [1, 4099, 1_048_579, 5_000_001])
@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_groupby_small_domain_additive_tables(n, case):
    kind, aggs = ADD_CASES[case]
    t = _table(n, 1200 + n + case)
    t["a32"] = (t["a8"].astype(np.int32) & 31).astype(np.int8)
    t["g6"] = (t["u8"] % 6).astype(np.uint8)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w", "a32", "g6"]
    cols = [cu(t[k]) for k in names]
    cols[4] = ops.Col(cols[4], 0, 2)
    cols[5] = ops.Col(cols[5], -2, 2)
    cols[8] = ops.Col(cols[8], 0, 31)
    cols[9] = ops.Col(cols[9], 0, 5)
    keys = {"a32": [8], "k12": [4, 5], "g6": [9]}[kind]
    out = ops.groupby_agg(cols, keys, aggs, preds=[(2, "<", 700)], strategy="small_domain")
    ops.check(out["status"])
    sel = R.filter([(t["b32"], "<", 700)], n)
    oa = [(op, t[names[a]] if a is not None else None, t[names[b]] if b is not None else None, kk)
          for op, a, b, kk in aggs]
    rk, ra = R.groupby([t[names[k]] for k in keys], oa, n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    for j in range(len(keys)):
        assert np.array_equal(np_(out["keys"][j], g), rk[:, j])
    for j in range(len(aggs)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), aggs[j]


def test_groupby_small_domain_additive_tables_device_count_and_unaligned_column():
    n, m = 3_000_000, 2_000_123
    aggs = ADD_CASES[2][1]
    t = _table(n, 78)
    t["g6"] = (t["u8"] % 6).astype(np.uint8)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w", "g6"]
    oa = [(op, t[names[a]] if a is not None else None, t[names[b]] if b is not None else None, kk)
          for op, a, b, kk in aggs]
    sel = R.filter([(t["b32"][:m], "<", 700)], m)
    rk, ra = R.groupby([t["g6"][:m]], oa, m, sel=sel)
    for unaligned in (False, True):
        cols = [cu(t[k]) for k in names]
        if unaligned:  # an 8-byte offset on an aggregate column: scalar loads
            buf = torch.zeros(n + 1, dtype=torch.int64, device=DEV)
            buf[1:] = cols[6]
            cols[6] = buf[1:]
            assert cols[6].data_ptr() % 16 == 8
        cols[8] = ops.Col(cols[8], 0, 5)
        nsel = torch.tensor([m], dtype=torch.int64, device=DEV)
        out = ops.groupby_agg(cols, [8], aggs, preds=[(2, "<", 700)], n=n, nsel=nsel, strategy="small_domain")
        ops.check(out["status"])
        g = int(out["ngroups"].item())
        assert g == len(rk)
        assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
        for j in range(len(aggs)):
            assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), (unaligned, aggs[j])


@pytest.mark.parametrize("n", [1, 4099, 300001])
def test_groupby_partition_large_domain(n):
    """PARTITION over domains of many buckets: one bounded int32 key over
    [-5M, 5M] (2442 buckets of 4096 gids), and two keys (int32 x int8) whose
    product spans 256 x 20001 gids; six aggregates, so narrower buckets; a
    row-list input; and a dense input cut by a device row count."""
    t = _table(n, 900 + n)
    r = np.random.default_rng(n)
    t["big"] = r.integers(-5_000_000, 5_000_001, n).astype(np.int32)
    t["mid"] = r.integers(-10000, 10001, n).astype(np.int32)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w", "big", "mid"]
    cols = [cu(t[k]) for k in names]
    cols[8] = ops.Col(cols[8], -5_000_000, 5_000_000)
    cols[9] = ops.Col(cols[9], -10000, 10000)
    cols[0] = ops.Col(cols[0], -128, 127)
    oaggs = _oracle_aggs(t, names)
    # one key, two aggregates (4096-gid buckets)
    out = ops.groupby_agg(cols, [8], [("sum", 6), ("count",)], strategy="partition")
    ops.check(out["status"])
    rk, ra = R.groupby([t["big"]], [("sum", t["v"], None, None), ("count", None, None, None)], n)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["aggs"][0], g), ra[:, 0])
    assert np.array_equal(np_(out["aggs"][1], g), ra[:, 1])
    # two keys, six aggregates, row list
    sel = R.filter([(t["c64"], ">", 0)], n)
    out = ops.groupby_agg(cols, [9, 0], AGGS6, sel=cu(sel), strategy="partition")
    ops.check(out["status"])
    rk, ra = R.groupby([t["mid"], t["a8"]], oaggs, n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["keys"][1], g), rk[:, 1])
    for j in range(len(AGGS6)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), AGGS6[j]
    # dense input limited by a device row count, with a fused filter
    m = n // 2 + 1
    d_n = torch.tensor([m], dtype=torch.int64, device=DEV)
    out = ops.groupby_agg(cols, [8], AGGS6, preds=[(2, ">=", 0)], nsel=d_n, strategy="partition")
    ops.check(out["status"])
    sel2 = R.filter([(t["b32"][:m], ">=", 0)], m)
    rk, ra = R.groupby([t["big"]], oaggs, n, sel=sel2)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    for j in range(len(AGGS6)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), AGGS6[j]


def test_groupby_partition_flags_keys_out_of_bounds_and_capacity():
    n = 50000
    t = _table(n, 4)
    t["big"] = np.random.default_rng(4).integers(0, 1_000_000, n).astype(np.int32)
    cols = [cu(t["big"]), cu(t["v"])]
    bounded = [ops.Col(cols[0], 0, 499_999), cols[1]]  # about half the keys lie above the bound
    out = ops.groupby_agg(bounded, [0], [("sum", 1)], strategy="partition")
    assert int(out["status"].item()) & 32  # TDP_ERR_OVERFLOW: rows out of bounds are dropped
    keep = np.flatnonzero(t["big"] <= 499_999).astype(np.int32)
    rk, ra = R.groupby([t["big"]], [("sum", t["v"], None, None)], n, sel=keep)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["aggs"][0], g), ra[:, 0])
    full = [ops.Col(cols[0], 0, 999_999), cols[1]]
    cap = 1000
    out = ops.groupby_agg(full, [0], [("sum", 1)], strategy="partition", capacity=cap)
    assert int(out["status"].item()) & 4  # TDP_ERR_CAPACITY
    rk, ra = R.groupby([t["big"]], [("sum", t["v"], None, None)], n)
    assert int(out["ngroups"].item()) == len(rk)
    assert np.array_equal(np_(out["keys"][0], cap), rk[:cap, 0])
    assert np.array_equal(np_(out["aggs"][0], cap), ra[:cap, 0])


@pytest.mark.parametrize("n", [5000, 300001])
def test_groupby_sort_unbounded_keys_and_row_list(n):
    """Sort strategy with keys without bounds (sign-flipped radix fields), a
    64-bit packed key (int32 + int8 + int32 = 72 bits is too wide, so use
    int32 + int8), and a row-id list input."""
    t = _table(n, 5 + n)
    t["b32"] = (t["b32"] // 7).astype(np.int32)  # many duplicates, negative keys
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    cols = [cu(t[k]) for k in names]
    sel = R.filter([(t["c64"], ">", 0)], n)
    out = ops.groupby_agg(cols, [2, 0], AGGS6, sel=cu(sel), strategy="sort")
    ops.check(out["status"])
    rk, ra = R.groupby([t["b32"], t["a8"]], _oracle_aggs(t, names), n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["keys"][1], g), rk[:, 1])
    for j in range(len(AGGS6)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j])


@pytest.mark.parametrize("agg", [("sum_mul_kminus", 6, 7, 100), ("avg", 6, None, None), ("min", 6, None, None),
                                 ("max", 6, None, None), ("sum", 6, None, None)])
def test_groupby_sort_single_value_aggregate(agg):
    """One value aggregate (+ COUNT): the sort carries the value itself."""
    n = 200003
    t = _table(n, 77)
    t["b32"] = (t["b32"] // 3).astype(np.int32)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    cols = [cu(t[k]) for k in names]
    out = ops.groupby_agg(cols, [2], [agg, ("count",)], strategy="sort")
    ops.check(out["status"])
    op, a, b, k = agg
    rk, ra = R.groupby([t["b32"]], [(op, t[names[a]], t[names[b]] if b is not None else None, k),
                                    ("count", None, None, None)], n)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"][0], g), rk[:, 0])
    assert np.array_equal(np_(out["aggs"][0], g), ra[:, 0])
    assert np.array_equal(np_(out["aggs"][1], g), ra[:, 1])


@pytest.mark.parametrize("n", [2_000_003, 6_000_001])
@pytest.mark.parametrize("case", ["few_groups", "many_groups", "carried_value"])
def test_groupby_sort_millions_of_rows(n, case):
    """Sort strategy over millions of rows behind a WHERE (the row count comes
    from the device).  The reduce spreads the sorted rows over hundreds of
    blocks: with 15 groups each group spans many warps' runs (slot values
    written into sorted order); with ~500K groups every run ends hundreds of
    groups (row ids carried through the sort); with one value aggregate the
    value itself is carried."""
    t = _table(n, 31 + n)
    names = ["a8", "u8", "b32", "c64", "k1", "k2", "v", "w"]
    cols = [cu(t[k]) for k in names]
    if case == "few_groups":
        cols[4] = ops.Col(cols[4], 0, 2)
        cols[5] = ops.Col(cols[5], -2, 2)
        keys, aggs, oaggs = [4, 5], AGGS6, _oracle_aggs(t, names)
    elif case == "many_groups":
        cols[2] = ops.Col(cols[2], -1000, 999)
        keys, aggs, oaggs = [2, 0], AGGS6, _oracle_aggs(t, names)
    else:
        keys = [2, 1]
        aggs = [("sum_mul_kminus", 6, 7, 100), ("count",)]
        oaggs = [("sum_mul_kminus", t["v"], t["w"], 100), ("count", None, None, None)]
    out = ops.groupby_agg(cols, keys, aggs, preds=[(3, ">", 0)], strategy="sort")
    ops.check(out["status"])
    sel = R.filter([(t["c64"], ">", 0)], n)
    rk, ra = R.groupby([t[names[k]] for k in keys], oaggs, n, sel=sel)
    g = int(out["ngroups"].item())
    assert g == len(rk)
    for j in range(len(keys)):
        assert np.array_equal(np_(out["keys"][j], g), rk[:, j])
    for j in range(len(aggs)):
        assert np.array_equal(np_(out["aggs"][j], g), ra[:, j]), aggs[j]


def test_groupby_config1_60k_both_strategies():
    n = 60000
    t = gen.fact_table(n, 15000, gen.BASE_SEED + 0)
    names = ["key", "flag", "status", "qty", "price", "disc", "date"]
    cols = [cu(t[k]) for k in names]
    cols[1] = ops.Col(cols[1], 0, 2)
    cols[2] = ops.Col(cols[2], 0, 1)
    aggs = [("sum", 3), ("sum", 4), ("sum_mul_kminus", 4, 5, 100), ("count",), ("avg", 3)]
    sel = R.filter([(t["date"], "<=", 2460)], n)
    rk, ra = R.groupby([t["flag"], t["status"]],
                       [("sum", t["qty"], None, None), ("sum", t["price"], None, None),
                        ("sum_mul_kminus", t["price"], t["disc"], 100), ("count", None, None, None),
                        ("avg", t["qty"], None, None)], n, sel=sel)
    for strategy in ("small_domain", "sort"):
        out = ops.groupby_agg(cols, [1, 2], aggs, preds=[(6, "<=", 2460)], strategy=strategy)
        ops.check(out["status"])
        g = int(out["ngroups"].item())
        assert g == 6
        assert np.array_equal(np.stack([np_(k, g) for k in out["keys"]], 1), rk)
        assert np.array_equal(np.stack([np_(a, g) for a in out["aggs"]], 1), ra)


def test_groupby_config1_60m_invariants():
    n = 60_000_000
    t = gen.fact_table(n, 15_000_000, gen.BASE_SEED + 1, cols=("flag", "status", "qty", "price", "disc", "date"))
    names = ["flag", "status", "qty", "price", "disc", "date"]
    cols = [cu(t[k]) for k in names]
    cols[0] = ops.Col(cols[0], 0, 2)
    cols[1] = ops.Col(cols[1], 0, 1)
    aggs = [("count",), ("sum", 2), ("sum_mul_kminus", 3, 4, 100)]
    out = ops.groupby_agg(cols, [0, 1], aggs, preds=[(5, "<=", 2460)], strategy="small_domain")
    ops.check(out["status"])
    keep = t["date"] <= 2460
    g = int(out["ngroups"].item())
    cnt, sq, sdp = (np_(a, g) for a in out["aggs"])
    assert cnt.sum() == keep.sum()
    assert sq.sum() == t["qty"][keep].sum()
    assert sdp.sum() == (t["price"][keep] * (100 - t["disc"][keep])).sum()
    # per-group sample: group (flag=1, status=0) one by one
    m = keep & (t["flag"] == 1) & (t["status"] == 0)
    j = 2 * 1 + 0
    assert cnt[j] == m.sum() and sq[j] == t["qty"][m].sum()


@pytest.mark.parametrize("n,bits", [(0, 8), (1, 8), (4096, 3), (4097, 24), (200000, 24), (123457, 64), (50000, 40)])
def test_sort_pairs_matches_oracle(n, bits):
    r = np.random.default_rng(n + bits)
    hi = (1 << bits) if bits < 64 else (1 << 63)
    keys = r.integers(0, hi, n, dtype=np.uint64) if bits < 64 else r.integers(0, 2**63, n).astype(np.uint64) * 2 + (r.integers(0, 2, n).astype(np.uint64))
    if n > 10:
        keys[: n // 3] = keys[0]  # long run of equal keys (stability)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, st = ops.sort_pairs(cu(keys.view(np.int64)), cu(vals.view(np.int32)), key_bits=bits)
    ops.check(st)
    ek, ev = R.sort_pairs(keys, vals)
    assert np.array_equal(np_(ko).view(np.uint64), ek)
    assert np.array_equal(np_(vo).view(np.uint32), ev)


def test_sort_pairs_unaligned_keys_and_skewed_digits():
    """Keys that start 8 bytes past a 16-byte boundary (the histogram reads
    them one by one) and digits that are mostly equal (runs of one digit
    within each lane's keys)."""
    n = 300001
    r = np.random.default_rng(17)
    keys = np.zeros(n + 1, np.uint64)
    keys[1:] = r.integers(0, 1 << 20, n, dtype=np.uint64)
    keys[1 : n // 2 + 1] &= 0xF00FF  # skewed: the middle digit is 0 for half the keys
    vals = r.integers(0, 2**31, n, dtype=np.uint32)
    k_all = cu(keys.view(np.int64))
    assert k_all[1:].data_ptr() % 16 != 0
    ko, vo, st = ops.sort_pairs(k_all[1:], cu(vals.view(np.int32)), key_bits=20)
    ops.check(st)
    ek, ev = R.sort_pairs(keys[1:], vals)
    assert np.array_equal(np_(ko).view(np.uint64), ek)
    assert np.array_equal(np_(vo).view(np.uint32), ev)


@pytest.mark.parametrize("nb,np_rows", [(1, 1), (1000, 5000), (300000, 1000003)])
def test_join_matches_oracle(nb, np_rows):
    r = np.random.default_rng(nb)
    bkey = (r.permutation(nb) * 2 + 1).astype(np.int32)
    bseg = r.integers(0, 5, nb).astype(np.int8)
    bpay = r.integers(-10**6, 10**6, nb).astype(np.int32)
    pkey = r.integers(0, 2 * nb + 2, np_rows).astype(np.int32)
    pdate = r.integers(0, 2557, np_rows).astype(np.int32)
    pval = r.integers(0, 10**9, np_rows).astype(np.int64)
    bcols = [cu(bkey), cu(bseg), cu(bpay)]
    pcols = [cu(pkey), cu(pdate), cu(pval)]
    table, st = ops.join_build(bcols, 0, payload_col=2, preds=[(1, "==", 2)])
    out = ops.join_probe(table, pcols, 0, preds=[(1, ">", 1200)], gather=[2], status=st)
    ops.check(st)
    bsel = R.filter([(bseg, "==", 2)], nb)
    psel = R.filter([(pdate, ">", 1200)], np_rows)
    op_, ob_, dup = R.join(bkey, pkey, bsel=bsel, psel=psel)
    assert not dup
    c = int(out["count"].item())
    assert c == len(op_)
    assert np.array_equal(np_(out["probe_row"], c), op_)
    assert np.array_equal(np_(out["payload"], c), bpay[ob_])
    assert np.array_equal(np_(out["gathered"][0], c), pval[op_])
    # one-call join without payload column: payload = build row id
    out2 = ops.join([cu(bkey)], 0, [cu(pkey)], 0)
    ops.check(out2["status"])
    op2, ob2, _ = R.join(bkey, pkey)
    c2 = int(out2["count"].item())
    assert c2 == len(op2)
    assert np.array_equal(np_(out2["probe_row"], c2), op2)
    assert np.array_equal(np_(out2["payload"], c2), ob2)


@pytest.mark.parametrize("nb,nslots", [(1000, 2048), (1000, 1024), (4000, 4096), (7, 8)])
def test_join_crowded_tables_walk_past_full_buckets(nb, nslots):
    """Load factors up to 1 (every bucket full): lookups continue into the
    following buckets, hits and misses both, including the wrap-around from
    the last bucket to the first."""
    r = np.random.default_rng(nslots + nb)
    bkey = r.choice(np.arange(-10**6, 10**6, dtype=np.int32), nb, replace=False)
    bpay = r.integers(-10**6, 10**6, nb).astype(np.int32)
    pkey = np.concatenate([bkey, r.integers(-10**6, 10**6, 3 * nb).astype(np.int32)])
    r.shuffle(pkey)
    table, st = ops.join_build([cu(bkey), cu(bpay)], 0, payload_col=1, nslots=nslots)
    out = ops.join_probe(table, [cu(pkey)], 0, gather=[0], status=st)
    ops.check(st)
    op_, ob_, dup = R.join(bkey, pkey)
    assert not dup
    c = int(out["count"].item())
    assert c == len(op_)
    assert np.array_equal(np_(out["probe_row"], c), op_)
    assert np.array_equal(np_(out["payload"], c), bpay[ob_])
    assert np.array_equal(np_(out["gathered"][0], c), pkey[op_])


def test_join_int32_min_key_is_flagged_and_never_found():
    imin = np.iinfo(np.int32).min
    bkey = np.array([3, imin, 5], np.int32)
    table, st = ops.join_build([cu(bkey)], 0)
    assert int(st.item()) == 32  # TDP_ERR_OVERFLOW only
    pkey = np.array([imin, 5, 3, imin, 4], np.int32)
    st2 = ops.new_status(DEV)
    out = ops.join_probe(table, [cu(pkey)], 0, status=st2)
    ops.check(st2)
    c = int(out["count"].item())
    assert c == 2
    assert np.array_equal(np_(out["probe_row"], c), [1, 2])
    assert np.array_equal(np_(out["payload"], c), [2, 0])


def test_join_duplicate_keys_and_full_table_are_flagged():
    bkey = cu(np.array([5, 7, 5, 9], np.int32))
    table, st = ops.join_build([bkey], 0)
    assert int(st.item()) & 8
    big = cu(np.arange(100, dtype=np.int32))
    table, st = ops.join_build([big], 0, nslots=64)
    assert int(st.item()) & 4
    with pytest.raises(TdpError):
        ops.join_build([big], 0, nslots=63)


@pytest.mark.parametrize("nslots", [None, 65536])  # default load <= 1/2; a dense table at load 0.76
def test_join_probe_agg_matches_join_then_groupby(nslots):
    nb, npr = 50000, 400000
    d = gen.chain_tables(npr, nb, 5000, seed=9, n_category=1000)
    cols_b = [cu(d["build_pk"]), cu(d["third_cat"][:nb] if len(d["third_cat"]) >= nb else np.resize(d["third_cat"], nb))]
    cat = cols_b[1].cpu().numpy()
    table, st = ops.join_build(cols_b, 0, payload_col=1, nslots=nslots)
    pcols = [cu(d["probe_fk"].astype(np.int32)), cu(d["probe_payload"])]
    out = ops.join_probe_agg(table, pcols, 0, 0, 999, [("sum", 1), ("count",)], status=st)
    ops.check(st)
    op_, ob_, _ = R.join(d["build_pk"], d["probe_fk"].astype(np.int32))
    g_cat = cat[ob_]
    rk, ra = R.groupby([g_cat.astype(np.int32)], [("sum", d["probe_payload"][op_], None, None),
                                                  ("count", None, None, None)], len(op_))
    g = int(out["ngroups"].item())
    assert g == len(rk)
    assert np.array_equal(np_(out["keys"], g), rk[:, 0])
    assert np.array_equal(np_(out["aggs"][0], g), ra[:, 0])
    assert np.array_equal(np_(out["aggs"][1], g), ra[:, 1])


@pytest.mark.parametrize("n,k", [(1, 1), (5, 10), (1000, 10), (2_600_000, 10), (300000, 16)])
def test_topk_matches_oracle(n, k):
    r = np.random.default_rng(n)
    vals = r.integers(-50, 50, n).astype(np.int64)  # many ties
    keys = r.permutation(n).astype(np.int32)
    ov, okk, dk = ops.topk(cu(vals), cu(keys), k)
    ev, ek = R.topk(vals, keys.astype(np.int64), k)
    m = int(dk.item())
    assert m == len(ev)
    assert np.array_equal(np_(ov, m), ev) and np.array_equal(np_(okk, m), ek)


def test_bounded_wait_times_out_without_hanging():
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = ops.new_status(DEV)
    ops.debug_wait_flag(flag, 1000, st)
    assert int(st.item()) == 16
    flag.fill_(1)
    st.zero_()
    ops.debug_wait_flag(flag, 1000, st)
    assert int(st.item()) == 0


def test_relational_results_are_deterministic():
    """Five runs of the shipping-priority plan give bitwise identical results."""
    from paper_2211_02753_b300 import plans
    nf, nd = 2_000_000, 500_000
    fact = {k: cu(v) for k, v in gen.fact_table(nf, nd, 5, cols=("key", "price", "disc", "date")).items()}
    dim = {k: cu(v) for k, v in gen.dim_table(nd, 5, cols=("key", "segment")).items()}
    p = plans.ShippingPriority(fact, dim)
    ref = None
    for _ in range(5):
        o = p.run()
        g = int(o["ngroups"].item())
        got = (np_(o["groups"]["keys"][0], g).tobytes(), np_(o["groups"]["aggs"][0], g).tobytes(),
               np_(o["top_vals"]).tobytes(), np_(o["top_keys"]).tobytes())
        ref = ref or got
        assert got == ref
    ops.check(p.status)


def test_shipping_plan_graph_replay_matches_eager():
    """The plan captured as a CUDA graph (the bench's timed step) gives the
    eager plan's results, and a replay reads new data copied into the
    plan's input tensors."""
    from paper_2211_02753_b300 import plans
    nf, nd = 2_000_000, 500_000
    fact = {k: cu(v) for k, v in gen.fact_table(nf, nd, 5, cols=("key", "price", "disc", "date")).items()}
    dim = {k: cu(v) for k, v in gen.dim_table(nd, 5, cols=("key", "segment")).items()}
    p = plans.ShippingPriority(fact, dim)

    def result(o):
        g = int(o["ngroups"].item())
        return (int(o["nmatch"].item()), np_(o["groups"]["keys"][0], g).tobytes(),
                np_(o["groups"]["aggs"][0], g).tobytes(), np_(o["top_vals"]).tobytes(), np_(o["top_keys"]).tobytes())

    ref = result(p.run())
    step = plans.Graphed(p)
    for _ in range(2):
        assert result(step.run()) == ref
    fact2 = gen.fact_table(nf, nd, 6, cols=("key", "price", "disc", "date"))
    for k in fact:
        fact[k].copy_(cu(fact2[k]))
    got = result(step.run())
    assert got != ref and got == result(p.run())
    ops.check(p.status)


# ------------------------------------------------------------ group-join

def _groupjoin_case(nb, npr, seed, lo, hi, key_span=None):
    r = np.random.default_rng(seed)
    span = hi - lo + 1
    bkey = (lo + r.permutation(span)[:nb]).astype(np.int32)
    bseg = r.integers(0, 5, nb).astype(np.int8)
    ks = key_span or (lo - 3, hi + 3)
    pkey = r.integers(ks[0], ks[1] + 1, npr).astype(np.int32)  # some keys outside the bounds
    pdate = r.integers(0, 2557, npr).astype(np.int32)
    pflag = r.integers(0, 3, npr).astype(np.int8)
    pv = r.integers(-10**9, 10**9, npr).astype(np.int64)
    pw = r.integers(0, 11, npr).astype(np.int64)
    p32 = r.integers(-1000, 1000, npr).astype(np.int32)
    return bkey, bseg, pkey, pdate, pflag, pv, pw, p32


GJ_AGGS = [("sum_mul_kminus", 4, 5, 100), ("count",), ("sum", 6), ("min", 4), ("max", 6), ("avg", 4)]


def _groupjoin_oracle(bkey, bseg, pkey, pdate, pflag, pv, pw, p32, nb, npr):
    bsel = R.filter([(bseg, "==", 2)], nb)
    psel = R.filter([(pdate, ">", 1200), (pflag, "!=", 1)], npr)
    prow, _, dup = R.join(bkey, pkey, bsel=bsel, psel=psel)
    assert not dup
    keys, aggs = R.groupby([pkey], [("sum_mul_kminus", pv, pw, 100), ("count", None, None, None),
                                    ("sum", p32, None, None), ("min", pv, None, None), ("max", p32, None, None),
                                    ("avg", pv, None, None)], npr, sel=prow)
    return len(prow), keys[:, 0], aggs


@pytest.mark.parametrize("nb,npr,lo,hi", [(0, 1000, 1, 100), (1, 1, 5, 5), (700, 0, -300, 1000),
                                          (5000, 70001, 1, 20000), (300000, 1_000_003, -1_500_000, 1_500_000),
                                          (32, 4097, 0, 31), (33, 4095, 7, 40)])
def test_groupjoin_matches_join_then_groupby(nb, npr, lo, hi):
    """JOIN ... GROUP BY key over the rank-coded build side equals the
    oracle's join followed by its group-by, for every aggregate, including
    empty sides, a one-key domain, a domain of exactly one bitmap word and
    ragged tiles of the probe."""
    bkey, bseg, pkey, pdate, pflag, pv, pw, p32 = _groupjoin_case(nb, npr, nb + npr, lo, hi)
    bcols = [cu(bkey), cu(bseg)]
    pcols = [cu(pkey), cu(pdate), cu(pflag), cu(pkey), cu(pv), cu(pw), cu(p32)]
    out = ops.groupjoin(bcols, 0, pcols, 0, lo, hi, GJ_AGGS, build_preds=[(1, "==", 2)],
                        probe_preds=[(1, ">", 1200), (2, "!=", 1)])
    ops.check(out["status"])
    nm, ek, ea = _groupjoin_oracle(bkey, bseg, pkey, pdate, pflag, pv, pw, p32, nb, npr)
    g = int(out["ngroups"].item())
    assert int(out["nmatch"].item()) == nm
    assert g == len(ek)
    assert np.array_equal(np_(out["keys"][0], g), ek)
    for j in range(len(GJ_AGGS)):
        assert np.array_equal(np_(out["aggs"][j], g), ea[:, j]), GJ_AGGS[j]


def test_groupjoin_unaligned_columns_counts_and_capacity():
    """Probe columns that do not start on a 16-byte boundary take the plain
    load path; d_n limits of both sides; an undersized output keeps the true
    group count and flags capacity."""
    nb, npr, lo, hi = 40000, 300001, 1, 60000
    bkey, bseg, pkey, pdate, pflag, pv, pw, p32 = _groupjoin_case(nb, npr + 1, 77, lo, hi)
    kdev = cu(pkey)[1:]  # 4-byte offset
    ddev = cu(pdate)[1:]
    pcols = [kdev, ddev, cu(pflag)[1:], kdev, cu(pv)[1:], cu(pw)[1:], cu(p32)[1:]]
    bcols = [cu(bkey), cu(bseg)]
    nb_lim, np_lim = 25000, 200000
    dnb = torch.tensor([nb_lim], dtype=torch.int64, device=DEV)
    dnp = torch.tensor([np_lim], dtype=torch.int64, device=DEV)
    out = ops.groupjoin(bcols, 0, pcols, 0, lo, hi, GJ_AGGS, build_preds=[(1, "==", 2)],
                        probe_preds=[(1, ">", 1200), (2, "!=", 1)], d_nbuild=dnb, d_nprobe=dnp)
    ops.check(out["status"])
    sl = slice(1, 1 + np_lim)
    nm, ek, ea = _groupjoin_oracle(bkey[:nb_lim], bseg[:nb_lim], pkey[sl], pdate[sl], pflag[sl], pv[sl], pw[sl],
                                   p32[sl], nb_lim, np_lim)
    g = int(out["ngroups"].item())
    assert int(out["nmatch"].item()) == nm and g == len(ek)
    assert np.array_equal(np_(out["keys"][0], g), ek)
    for j in range(len(GJ_AGGS)):
        assert np.array_equal(np_(out["aggs"][j], g), ea[:, j])
    cap = g // 2
    small = ops.groupjoin(bcols, 0, pcols, 0, lo, hi, GJ_AGGS, build_preds=[(1, "==", 2)],
                          probe_preds=[(1, ">", 1200), (2, "!=", 1)], d_nbuild=dnb, d_nprobe=dnp, capacity=cap)
    assert int(small["status"].item()) == 4
    assert int(small["ngroups"].item()) == g
    assert np.array_equal(np_(small["keys"][0], cap), ek[:cap])
    assert np.array_equal(np_(small["aggs"][0], cap), ea[:cap, 0])


def test_groupjoin_flags_duplicate_and_out_of_bounds_build_keys():
    bkey = cu(np.array([5, 7, 5, 9], np.int32))
    pk = cu(np.array([5, 7, 9, 11], np.int32))
    pv = cu(np.array([1, 2, 3, 4], np.int64))
    out = ops.groupjoin([bkey], 0, [pk, pv], 0, 0, 20, [("sum", 1)])
    assert int(out["status"].item()) & 8
    bkey2 = cu(np.array([5, 70, 9], np.int32))  # 70 is outside [0, 20]
    out2 = ops.groupjoin([bkey2], 0, [pk, pv], 0, 0, 20, [("sum", 1)])
    assert int(out2["status"].item()) == 32
    g = int(out2["ngroups"].item())
    assert g == 2
    assert np_(out2["keys"][0], g).tolist() == [5, 9]
    assert np_(out2["aggs"][0], g).tolist() == [1, 3]
    with pytest.raises(TdpError):
        ops.groupjoin([bkey], 0, [pk, pv], 0, 20, 0, [("sum", 1)])


@pytest.mark.parametrize("nb", [1, 15, 16, 17, 100_003])
def test_groupjoin_build_predicates_every_column_type(nb):
    """Build-side filters on uint8, int8, int32 and int64 columns (the 16-row
    vector path and the ragged tail) select the same build keys as the
    oracle's filter."""
    r = np.random.default_rng(nb)
    lo, hi = -50, 3 * nb + 50
    bkey = (lo + r.permutation(hi - lo + 1)[:nb]).astype(np.int32)
    u8 = r.integers(0, 256, nb).astype(np.uint8)
    i8 = r.integers(-128, 128, nb).astype(np.int8)
    i32 = r.integers(-1000, 1000, nb).astype(np.int32)
    i64 = r.integers(-10**12, 10**12, nb).astype(np.int64)
    npr = 4 * nb + 7
    pkey = r.integers(lo - 5, hi + 5, npr).astype(np.int32)
    pv = r.integers(0, 10**6, npr).astype(np.int64)
    preds = [(1, "<", 200), (2, "!=", -3), (3, ">=", -700), (4, "<=", 5 * 10**11)]
    out = ops.groupjoin([cu(bkey), cu(u8), cu(i8), cu(i32), cu(i64)], 0, [cu(pkey), cu(pv)], 0, lo, hi,
                        [("sum", 1), ("count",)], build_preds=preds)
    ops.check(out["status"])
    cols = [bkey, u8, i8, i32, i64]
    bsel = R.filter([(cols[c], op, lit) for c, op, lit in preds], nb)
    prow, _, _ = R.join(bkey, pkey, bsel=bsel)
    keys, aggs = R.groupby([pkey], [("sum", pv, None, None), ("count", None, None, None)], npr, sel=prow)
    g = int(out["ngroups"].item())
    assert g == len(keys) and int(out["nmatch"].item()) == len(prow)
    assert np.array_equal(np_(out["keys"][0], g), keys[:, 0])
    assert np.array_equal(np_(out["aggs"][0], g), aggs[:, 0])
    assert np.array_equal(np_(out["aggs"][1], g), aggs[:, 1])


@pytest.mark.parametrize("k", [1, 10, 16])
def test_groupjoin_fused_topk_matches_oracle_topk(k):
    """The fused ORDER BY ... LIMIT k over the groups (ties broken by key)
    equals the oracle's top-k of the oracle's groups; few groups (fewer than
    k) and heavy ties included."""
    for nb, npr, span in ((5, 40, 3), (20000, 300000, 50), (200000, 2_000_000, 10**6)):
        r = np.random.default_rng(nb + k)
        bkey = (1 + r.permutation(4 * nb)[:nb]).astype(np.int32)
        pkey = r.integers(1, 4 * nb + 1, npr).astype(np.int32)
        pv = r.integers(0, span, npr).astype(np.int64)  # small spans: many equal sums
        out = ops.groupjoin([cu(bkey)], 0, [cu(pkey), cu(pv)], 0, 1, 4 * nb, [("sum", 1)], topk=k, topk_agg=0)
        ops.check(out["status"])
        prow, _, _ = R.join(bkey, pkey)
        keys, aggs = R.groupby([pkey], [("sum", pv, None, None)], npr, sel=prow)
        ev, ek = R.topk(aggs[:, 0], keys[:, 0], k)
        m = int(out["k"].item())
        assert m == len(ev)
        assert np.array_equal(np_(out["top_vals"], m), ev)
        assert np.array_equal(np_(out["top_keys"], m), ek)


def test_groupjoin_widest_key_domain():
    """A key domain of 2^31 values (the largest the call takes): the bitmap
    has more words than the resident blocks cover at once, so the rank and
    finalize passes take several spans per block; keys at both ends of the
    domain and probe keys outside it."""
    lo, hi = -(1 << 30), (1 << 30) - 1
    r = np.random.default_rng(2031)
    nb, npr = 100_000, 1_000_000
    bkey = np.unique(r.integers(lo, hi + 1, nb + 1000, dtype=np.int64))[:nb]
    bkey[0], bkey[-1] = lo, hi
    r.shuffle(bkey)
    bkey = bkey.astype(np.int32)
    pkey = np.concatenate([r.choice(bkey, npr // 2), r.integers(np.iinfo(np.int32).min, np.iinfo(np.int32).max,
                                                                  npr // 2, dtype=np.int64)]).astype(np.int32)
    pkey[:3] = [lo, hi, lo - 1]
    pv = r.integers(-10**9, 10**9, npr).astype(np.int64)
    out = ops.groupjoin([cu(bkey)], 0, [cu(pkey), cu(pv)], 0, lo, hi, [("sum", 1), ("count",), ("max", 1)],
                        topk=5, topk_agg=0)
    ops.check(out["status"])
    prow, _, _ = R.join(bkey, pkey)
    keys, aggs = R.groupby([pkey], [("sum", pv, None, None), ("count", None, None, None), ("max", pv, None, None)],
                           npr, sel=prow)
    g = int(out["ngroups"].item())
    assert g == len(keys) and int(out["nmatch"].item()) == len(prow)
    assert np.array_equal(np_(out["keys"][0], g), keys[:, 0])
    for j in range(3):
        assert np.array_equal(np_(out["aggs"][j], g), aggs[:, j])
    ev, ek = R.topk(aggs[:, 0], keys[:, 0], 5)
    assert np.array_equal(np_(out["top_vals"], 5), ev) and np.array_equal(np_(out["top_keys"], 5), ek)


def test_groupjoin_steps_with_several_probe_batches():
    """build once, probe three batches (their own columns, each with its own
    fused filter), finish: equal to one probe over the concatenated rows, and
    to the oracle; the same object reused for a second round gives the same
    result (the build step clears the workspace)."""
    lo, hi, nb, npr = 1, 50000, 20000, 600_001
    bkey, bseg, pkey, pdate, pflag, pv, pw, p32 = _groupjoin_case(nb, npr, 41, lo, hi)
    aggs = [("sum_mul_kminus", 4, 5, 100), ("count",), ("avg", 4)]
    gj = ops.GroupJoin(nb, lo, hi, aggs, topk=7, topk_agg=0, device=DEV)
    cuts = [0, 150_000, 150_001, npr]
    for _ in range(2):
        gj.build([cu(bkey), cu(bseg)], 0, preds=[(1, "==", 2)])
        for a, b in zip(cuts[:-1], cuts[1:]):
            pc = [cu(pkey[a:b]), cu(pdate[a:b]), cu(pflag[a:b]), cu(pkey[a:b]), cu(pv[a:b]), cu(pw[a:b])]
            gj.probe(pc, 0, preds=[(1, ">", 1200), (2, "!=", 1)])
        out = gj.finish()
        torch.cuda.synchronize()
        bsel = R.filter([(bseg, "==", 2)], nb)
        psel = R.filter([(pdate, ">", 1200), (pflag, "!=", 1)], npr)
        prow, _, _ = R.join(bkey, pkey, bsel=bsel, psel=psel)
        keys, ea = R.groupby([pkey], [("sum_mul_kminus", pv, pw, 100), ("count", None, None, None),
                                      ("avg", pv, None, None)], npr, sel=prow)
        g = int(out["ngroups"].item())
        assert g == len(keys) and int(out["nmatch"].item()) == len(prow)
        assert np.array_equal(np_(out["keys"][0], g), keys[:, 0])
        for j in range(3):
            assert np.array_equal(np_(out["aggs"][j], g), ea[:, j])
        ev, ek = R.topk(ea[:, 0], keys[:, 0], 7)
        assert np.array_equal(np_(out["top_vals"], 7), ev) and np.array_equal(np_(out["top_keys"], 7), ek)
