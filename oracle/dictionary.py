"""Order-preserving dictionary encoding of a string column (Sec. 2, Data
Encoding: a string column is stored as codes of a dictionary whose order is
the strings' order).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The definition written out: the dictionary is the column's distinct strings
in ascending bytewise order (Python's ``bytes`` comparison: unsigned bytes,
a proper prefix before its extensions), and a row's code is its string's
position in that list.
"""
from __future__ import annotations

import numpy as np


def split(offsets, data):
    """The rows of an offsets + bytes string column as a list of bytes."""
    offsets = np.asarray(offsets, np.int64)
    data = np.asarray(data, np.uint8).tobytes()
    return [data[offsets[i]:offsets[i + 1]] for i in range(len(offsets) - 1)]


def dict_encode(strings):
    """Returns (codes int32[n], dictionary: list of bytes in ascending order)."""
    dictionary = sorted(set(strings))
    index = {s: i for i, s in enumerate(dictionary)}
    return np.array([index[s] for s in strings], dtype=np.int32), dictionary


def join_strings(strings):
    """The offsets + bytes layout (int32 offsets, uint8 data) of a list of bytes."""
    offsets = np.zeros(len(strings) + 1, np.int32)
    if strings:
        offsets[1:] = np.cumsum([len(s) for s in strings])
    data = np.frombuffer(b"".join(strings), dtype=np.uint8).copy() if strings else np.zeros(0, np.uint8)
    return offsets, data
