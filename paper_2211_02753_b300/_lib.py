"""ctypes loader for ``libtdp.so`` (the C ABI declared in include/tdp.h).

The library is built in-tree by ``paper_2211_02753_b300/build.py``.  There is
no fallback: if the shared library is missing or does not load, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdp.so")

# tdp_dtype
I8, U8, I32, I64, F32, BF16 = 0, 1, 2, 3, 4, 5
# tdp_cmp
CMP = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}
# tdp_agg_op
AGG = {"count": 0, "sum": 1, "sum_mul_kminus": 2, "avg": 3, "min": 4, "max": 5}
# tdp_groupby_strategy
STRATEGY = {"auto": 0, "sort": 1, "small_domain": 2, "partition": 3}
JOIN_UNIQUE_BUILD = 1

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported dtype", 3: "workspace too small",
          4: "capacity exceeded", 8: "duplicate build key", 16: "bounded device wait timed out",
          32: "arithmetic overflow", 64: "CUDA launch error"}


class TdpCol(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("has_bounds", C.c_int32),
                ("n", C.c_int64), ("lo", C.c_int64), ("hi", C.c_int64)]


class TdpPred(C.Structure):
    _fields_ = [("col", C.c_int32), ("cmp", C.c_int32), ("lit", C.c_int64)]


class TdpAgg(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("reserved", C.c_int32), ("k", C.c_int64)]


class TdpError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        names = [v for k, v in STATUS.items() if k and (self.status & k) == k] if self.status > 3 else \
            [STATUS.get(self.status, "unknown")]
        super().__init__("%s: tdp status %d (%s)" % (where or "tdp", self.status, ", ".join(names)))


_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_u32 = C.c_uint32
_sz = C.c_size_t
_f = C.c_float
_st = C.c_int32

# name -> (restype, argtypes)
SIGNATURES = {
    "tdp_status_str": (C.c_char_p, [_i32]),
    "tdp_abi_version": (_i32, []),
    "tdp_set_spin_limit": (_u32, [_u32]),
    "tdp_debug_wait_flag": (_st, [_p, _u32, _p, _p]),
    "tdp_filter_workspace": (_sz, [_i64]),
    "tdp_filter": (_st, [_p, _i32, _p, _i32, _i64, _p, _p, _i64, _p, _p, _i32, _p, _p, _sz, _p, _p]),
    "tdp_groupby_agg_workspace": (_sz, [_i64, _p, _i32, _i32, _i32]),
    "tdp_groupby_agg": (_st, [_p, _i32, _p, _i32, _i64, _p, _p, _p, _i32, _p, _i32, _i32, _p, _p, _i64, _p,
                              _p, _sz, _p, _p]),
    "tdp_sort_pairs_workspace": (_sz, [_i64, _i32]),
    "tdp_sort_pairs": (_st, [_p, _p, _i64, _i32, _p, _p, _p, _sz, _p, _p]),
    "tdp_join_default_slots": (_i64, [_i64]),
    "tdp_join_build": (_st, [_p, _i32, _p, _i32, _i64, _p, _i32, _i32, _u32, _p, _i64, _p, _p]),
    "tdp_join_probe_workspace": (_sz, [_i64]),
    "tdp_join_probe": (_st, [_p, _i64, _p, _i32, _p, _i32, _i64, _p, _p, _i32, _p, _p, _p, _i32, _p, _i64, _p,
                             _p, _sz, _p, _p]),
    "tdp_join_workspace": (_sz, [_i64, _i64, _i64]),
    "tdp_join": (_st, [_p, _i32, _p, _i32, _i64, _i32, _i32, _p, _i32, _p, _i32, _i64, _i32, _i64, _p, _p, _p,
                       _i32, _p, _i64, _p, _p, _sz, _p, _p]),
    "tdp_join_nm_workspace": (_sz, [_i64, _i64]),
    "tdp_join_nm": (_st, [_p, _i32, _p, _i32, _i64, _p, _i32, _p, _i32, _p, _i32, _i64, _p, _i32, _p, _p, _i64, _p,
                          _p, _sz, _p, _p]),
    "tdp_join_probe_agg_workspace": (_sz, [_i64, _i64, _i32]),
    "tdp_join_probe_agg": (_st, [_p, _i64, _p, _i32, _p, _i32, _i64, _p, _i32, _i64, _i64, _p, _i32, _p, _p,
                                 _i64, _p, _p, _sz, _p, _p]),
    "tdp_groupjoin_workspace": (_sz, [_i64, _i64, _i64, _i32, _i32]),
    "tdp_groupjoin": (_st, [_p, _i32, _p, _i32, _i64, _p, _i32, _p, _i32, _p, _i32, _i64, _p, _i32, _i64, _i64,
                            _p, _i32, _p, _p, _i64, _p, _p, _i32, _i32, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_groupjoin_build": (_st, [_p, _i32, _p, _i32, _i64, _p, _i32, _i64, _i64, _p, _i32, _i32, _p, _sz, _p, _p]),
    "tdp_groupjoin_probe": (_st, [_p, _i32, _p, _i32, _i64, _p, _i32, _i64, _i64, _i64, _p, _i32, _i32, _p, _sz, _p,
                                  _p]),
    "tdp_groupjoin_finish": (_st, [_i64, _i64, _i64, _p, _i32, _p, _p, _i64, _p, _p, _i32, _i32, _p, _p, _p, _p, _sz,
                                   _p, _p]),
    "tdp_dict_encode_workspace": (_sz, [_i64, _i32]),
    "tdp_dict_encode": (_st, [_p, _p, _i64, _i32, _p, _p, _p, _i64, _i64, _p, _p, _p, _sz, _p, _p]),
    "tdp_topk_workspace": (_sz, [_i64, _i32]),
    "tdp_topk": (_st, [_p, _p, _i64, _p, _i32, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_soft_workspace": (_sz, [_i64, _i32]),
    "tdp_soft_filter_fwd": (_st, [_p, _p, _p, _f, _i64, _p, _p]),
    "tdp_soft_filter_bwd": (_st, [_p, _p, _p, _f, _i64, _i32, _p, _p, _p, _p, _sz, _p]),
    "tdp_soft_agg_fwd": (_st, [_p, _p, _p, _p, _f, _i64, _i32, _p, _p, _p, _sz, _p]),
    "tdp_soft_agg_fwd_noalloc": (_st, [_p, _p, _p, _p, _f, _i64, _i32, _p, _p, _p]),
    "tdp_soft_agg_bwd": (_st, [_p, _p, _p, _p, _f, _i64, _i32, _p, _p, _p, _p, _p, _p, _sz, _p]),
    # glyph CNN of the trainable query (include/tdp_cnn.h)
    "tdp_cnn_conv1_fwd": (_st, [_p, _i64, _p, _p, _p, _p]),
    "tdp_cnn_conv2_pool_fwd": (_st, [_p, _i64, _p, _p, _p, _p, _p, _p]),
    "tdp_cnn_fc1_fwd_workspace": (_sz, [_i64]),
    "tdp_cnn_fc1_fwd": (_st, [_p, _i64, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_cnn_head_workspace": (_sz, [_i64]),
    "tdp_cnn_head": (_st, [_p, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "tdp_cnn_head2_workspace": (_sz, [_i64]),
    "tdp_cnn_head2": (_st, [_p, _i64] + [_p] * 17 + [_sz, _p]),
    "tdp_cnn_fc1_bwd_workspace": (_sz, [_i64]),
    "tdp_cnn_fc1_bwd": (_st, [_p, _p, _p, _i64, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_cnn_conv2_bwd_workspace": (_sz, [_i64]),
    "tdp_cnn_conv2_bwd": (_st, [_p, _p, _p, _p, _i64, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_cnn_conv1_bwd_workspace": (_sz, [_i64]),
    "tdp_cnn_conv1_bwd": (_st, [_p, _p, _i64, _p, _p, _p, _sz, _p]),
    "tdp_adam_step": (_st, [_p, _p, _p, _p, _p, _p, _i32, _i32, _f, _f, _f, _f, _p]),
    "tdp_f32_to_bf16": (_st, [_p, _i64, _p, _p]),
    "tdp_exact_pe_count": (_st, [_p, _i64, _i32, _i32, _i32, _p, _p, _p, _p]),
    "tdp_pe_groupby_fwd": (_st, [_p, _i64, _i32, _i32, _i32, _p, _p, _p]),
    "tdp_pe_groupby_bwd": (_st, [_p, _p, _i64, _i32, _i32, _i32, _p, _p]),
    # soft ORDER BY ... LIMIT k (include/tdp_softsort.h)
    "tdp_soft_topk_fwd": (_st, [_p, _p, _i64, _p, _i64, _i64, _i32, _f, _f, _p, _p, _p, _p, _p]),
    "tdp_soft_topk_workspace": (_sz, [_i64]),
    "tdp_soft_topk_bwd": (_st, [_p, _p, _i64, _p, _i64, _i64, _i32, _f, _f, _p, _p, _p, _p, _p, _p, _p, _sz, _p,
                                _p]),
    "tdp_exact_topk": (_st, [_p, _p, _i64, _p, _i64, _i64, _i32, _p, _p, _p, _p]),
    # learning from label proportions (include/tdp_llp.h)
    "tdp_llp_counts": (_st, [_p, _i64, _i32, _i64, _p, _f, _p, _p, _p]),
    "tdp_llp_step_workspace": (_sz, [_i64, _i32, _i32, _i64]),
    "tdp_llp_step": (_st, [_p, _i64, _i32, _i32, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p, _p]),
    "tdp_llp_predict": (_st, [_p, _i64, _i32, _i32, _p, _p, _p, _p, _p, _p]),
    "tdp_exact_pe_count2": (_st, [_p, _i32, _p, _i32, _i64, _i32, _p, _p, _p, _p]),
    "tdp_pe_groupby2_fwd": (_st, [_p, _i32, _p, _i32, _i64, _i32, _p, _p]),
    "tdp_pe_groupby2_bwd": (_st, [_p, _p, _i32, _p, _i32, _i64, _i32, _p, _p, _p]),
}

_lib = None


def lib():
    """The loaded library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtdp.so not built: run `python -m paper_2211_02753_b300.build` "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def call(name: str, *args):
    """Calls a status-returning entry point; raises TdpError on failure."""
    st = getattr(lib(), name)(*args)
    if st != 0:
        raise TdpError(st, name)
    return st
