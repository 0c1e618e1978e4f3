"""N:M equi-join and order-preserving dictionary codes on the GPU against
the oracle, bit-exact.

N:M join: every (probe row, build row) pair with equal keys in probe order,
then build-row order (oracle.relational.join, which sorts the build side and
binary-searches every probe key).  Dictionary codes: oracle.dictionary; a
multi-key GROUP BY over (string code, int column) against the oracle's
group-by over its own codes, with the group keys decoded back to strings."""
import numpy as np
import pytest
import torch

import gen
from oracle import dictionary as D
from oracle import relational as R
from paper_2211_02753_b300 import ops

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def np_(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


@pytest.mark.parametrize("nb,npr,dup", [(0, 100, 1.0), (1, 1, 1.0), (1000, 5000, 8.0), (4097, 10001, 1.0),
                                        (200_003, 1_000_001, 12.0), (50_000, 300_000, 400.0)])
def test_join_nm_matches_oracle(nb, npr, dup):
    d = gen.nm_join_tables(nb, npr, dup, seed=nb + npr)
    bseg = np.random.default_rng(nb).integers(0, 5, nb).astype(np.int8)
    bsel = R.filter([(bseg, "!=", 3)], nb)
    psel = R.filter([(d["probe_date"], ">", 1200)], npr)
    ep, eb, _ = R.join(d["build_key"], d["probe_key"], bsel=bsel, psel=psel)
    out = ops.join_nm([cu(d["build_key"]), cu(bseg)], 0, [cu(d["probe_key"]), cu(d["probe_date"])], 0,
                      build_preds=[(1, "!=", 3)], probe_preds=[(1, ">", 1200)], capacity=len(ep) + 16)
    ops.check(out["status"])
    c = int(out["count"].item())
    assert c == len(ep)
    assert np.array_equal(np_(out["probe_row"], c), ep)
    assert np.array_equal(np_(out["build_row"], c), eb)


def test_join_nm_workload_size():
    """The benchmark's N:M join: 10M build rows (about 12 per key), 20M probe
    rows behind date > 1200 -- about 63M pairs, every one compared."""
    d = gen.nm_join_tables(10_000_000, 20_000_000, 12.0, gen.BASE_SEED + 6)
    psel = R.filter([(d["probe_date"], ">", 1200)], 20_000_000)
    ep, eb, _ = R.join(d["build_key"], d["probe_key"], psel=psel)
    out = ops.join_nm([cu(d["build_key"])], 0, [cu(d["probe_key"]), cu(d["probe_date"])], 0,
                      probe_preds=[(1, ">", 1200)], capacity=len(ep) + 16)
    ops.check(out["status"])
    c = int(out["count"].item())
    assert c == len(ep)
    assert np.array_equal(np_(out["probe_row"], c), ep)
    assert np.array_equal(np_(out["build_row"], c), eb)


def test_join_nm_counts_capacity_and_int32_min():
    imin = np.iinfo(np.int32).min
    bkey = np.array([5, 7, 5, imin, 9, 5, 7], np.int32)
    pkey = np.array([5, imin, 7, 8, 5, 9], np.int32)
    out = ops.join_nm([cu(bkey)], 0, [cu(pkey)], 0, capacity=32)
    assert int(out["status"].item()) == 32  # the INT32_MIN build row is flagged and dropped
    ep, eb, _ = R.join(np.delete(bkey, 3), pkey)
    eb = np.where(eb >= 3, eb + 1, eb)  # build row ids of the original table
    c = int(out["count"].item())
    assert c == len(ep) == 9
    assert np.array_equal(np_(out["probe_row"], c), ep) and np.array_equal(np_(out["build_row"], c), eb)
    small = ops.join_nm([cu(bkey)], 0, [cu(pkey)], 0, capacity=4)
    assert int(small["status"].item()) & 4 and int(small["count"].item()) == 9
    assert np.array_equal(np_(small["probe_row"], 4), ep[:4])
    # d_n limits on both sides
    dnb = torch.tensor([3], dtype=torch.int64, device=DEV)
    dnp = torch.tensor([4], dtype=torch.int64, device=DEV)
    lim = ops.join_nm([cu(bkey)], 0, [cu(pkey)], 0, d_nbuild=dnb, d_nprobe=dnp, capacity=32)
    ops.check(lim["status"])
    ep2, eb2, _ = R.join(bkey[:3], pkey[:4])
    c2 = int(lim["count"].item())
    assert c2 == len(ep2) and np.array_equal(np_(lim["build_row"], c2), eb2)


def _dict_case(strings):
    off, data = D.join_strings(strings)
    return cu(off), cu(data if len(data) else np.zeros(1, np.uint8))


@pytest.mark.parametrize("n,words,max_len", [(1, 1, 8), (1000, 50, 8), (4097, 300, 16), (100_003, 5000, 24),
                                             (300_000, 20000, 32), (2_000_003, 1_500_000, 24)])
def test_dict_encode_matches_oracle(n, words, max_len):
    off, data, vocab, idx = gen.string_column(n, words, seed=n, max_len=max_len)
    strings = D.split(off, data)
    out = ops.dict_encode(cu(off), cu(data if len(data) else np.zeros(1, np.uint8)), max_len=max_len)
    ops.check(out["status"])
    ec, ed = D.dict_encode(strings)
    assert np.array_equal(np_(out["codes"], n), ec)
    nd, nbytes = int(out["ndict"].item()), int(out["nbytes"].item())
    assert nd == len(ed) and nbytes == sum(len(w) for w in ed)
    got = D.split(np_(out["dict_offsets"], nd + 1), np_(out["dict_bytes"], nbytes))
    assert got == ed


def test_dict_encode_workload_size():
    """The benchmark's column: 10M rows drawn from 100K words of up to 24
    bytes.  Every row is its vocabulary word, so the oracle encodes the words
    the rows use (the same strings, each once) and a row's expected code is
    its word's; the dictionary is compared whole."""
    off, data, vocab, idx = gen.string_column(10_000_000, 100_000, gen.BASE_SEED + 7, max_len=24)
    out = ops.dict_encode(cu(off), cu(data), max_len=24)
    ops.check(out["status"])
    used = np.unique(idx)
    wc, ed = D.dict_encode([vocab[u] for u in used])
    code_of_word = np.full(len(vocab), -1, np.int64)
    code_of_word[used] = wc
    assert np.array_equal(np_(out["codes"], len(idx)), code_of_word[idx])
    nd, nbytes = int(out["ndict"].item()), int(out["nbytes"].item())
    assert nd == len(ed) and nbytes == sum(len(w) for w in ed)
    assert D.split(np_(out["dict_offsets"], nd + 1), np_(out["dict_bytes"], nbytes)) == ed


def test_dict_encode_edge_strings():
    """The empty string, proper prefixes, bytes above 0x7f (unsigned order),
    strings that differ only in their last byte of a word, the longest
    allowed, and one over the limit (flagged, encoded as the empty string)."""
    s = [b"", b"a", b"ab", b"abcdefgh", b"abcdefgi", b"abcdefgh" + b"z", b"\xff", b"\x80\x01", b"\x7f",
         b"x" * 32, b"x" * 31, b"", b"ab", b"abcdefgh"]
    out = ops.dict_encode(*_dict_case(s), max_len=32)
    ops.check(out["status"])
    ec, ed = D.dict_encode(s)
    assert np.array_equal(np_(out["codes"], len(s)), ec)
    too_long = s + [b"y" * 33]
    out2 = ops.dict_encode(*_dict_case(too_long), max_len=32)
    assert int(out2["status"].item()) == 32
    ec2, _ = D.dict_encode(s + [b""])
    assert np.array_equal(np_(out2["codes"], len(too_long)), ec2)
    empty = ops.dict_encode(cu(np.zeros(1, np.int32)), cu(np.zeros(1, np.uint8)))
    ops.check(empty["status"])
    assert int(empty["ndict"].item()) == 0


def test_group_by_dictionary_code_and_flag():
    """GROUP BY (string, flag) with SUM, COUNT, AVG through the codes: the
    groups come out in (string, flag) order, equal to the oracle's group-by
    over its own codes, and decode back to the same strings."""
    n = 500_001
    off, data, vocab, idx = gen.string_column(n, 3000, seed=9, max_len=20)
    strings = D.split(off, data)
    r = np.random.default_rng(9)
    flag = r.integers(0, 3, n).astype(np.int8)
    price = r.integers(90000, 10500000, n).astype(np.int64)
    enc = ops.dict_encode(cu(off), cu(data), max_len=20)
    ops.check(enc["status"])
    nd = int(enc["ndict"].item())
    cols = [ops.Col(enc["codes"][:n], 0, nd - 1), ops.Col(cu(flag), 0, 2), cu(price)]
    aggs = [("sum", 2), ("count",), ("avg", 2)]
    for strategy in ("auto", "sort"):
        gb = ops.groupby_agg(cols, [0, 1], aggs, strategy=strategy)
        ops.check(gb["status"])
        ec, ed = D.dict_encode(strings)
        keys, ea = R.groupby([ec, flag], [("sum", price, None, None), ("count", None, None, None),
                                          ("avg", price, None, None)], n)
        g = int(gb["ngroups"].item())
        assert g == len(keys)
        gk = np.stack([np_(k, g).astype(np.int64) for k in gb["keys"]], 1)
        assert np.array_equal(gk, keys)
        for j in range(3):
            assert np.array_equal(np_(gb["aggs"][j], g), ea[:, j])
        dic = D.split(np_(enc["dict_offsets"], nd + 1), np_(enc["dict_bytes"], int(enc["nbytes"].item())))
        decoded = [(dic[c], f) for c, f in gk[:50]]
        assert decoded == sorted(decoded) == [(ed[c], f) for c, f in keys[:50]]
