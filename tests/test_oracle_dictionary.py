"""Pins of the dictionary-encoding oracle (Sec. 2, Data Encoding):
numpy's unique (a library routine) on the same strings, the order
preservation that defines the encoding, the round trip, and hand cases for
prefixes and the empty string."""
import numpy as np

import gen
from oracle import dictionary as D


def test_hand_cases_prefix_first_and_empty_string():
    s = [b"ab", b"", b"abc", b"b", b"ab", b"a", b"", b"abc", b"aa"]
    codes, d = D.dict_encode(s)
    assert d == [b"", b"a", b"aa", b"ab", b"abc", b"b"]
    assert codes.tolist() == [3, 0, 4, 5, 3, 1, 0, 4, 2]


def test_matches_numpy_unique_and_preserves_order():
    off, data, vocab, idx = gen.string_column(20000, 700, seed=5)
    s = D.split(off, data)
    assert s == [vocab[i] for i in idx]
    codes, d = D.dict_encode(s)
    uniq, inv = np.unique(np.array(s, dtype=object), return_inverse=True)
    assert list(uniq) == d and np.array_equal(inv.ravel(), codes)
    # order preservation and round trip on a sample of pairs
    r = np.random.default_rng(1)
    for i, j in r.integers(0, len(s), (2000, 2)):
        assert (codes[i] < codes[j]) == (s[i] < s[j])
        assert (codes[i] == codes[j]) == (s[i] == s[j])
    assert [d[c] for c in codes] == s


def test_join_split_round_trip():
    s = [b"x", b"", b"hello", b"hel"]
    off, data = D.join_strings(s)
    assert off.tolist() == [0, 1, 1, 6, 9]
    assert D.split(off, data) == s
