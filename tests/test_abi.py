"""The C-ABI library loads and exports every symbol the public headers declare
(no compute call: this runs without a GPU)."""
import glob
import os
import re

from paper_2211_02753_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tdp_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = _lib.lib()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # every declared function has a ctypes signature in the binding
    assert names <= set(_lib.SIGNATURES), sorted(names - set(_lib.SIGNATURES))


def test_host_only_calls():
    L = _lib.lib()
    assert L.tdp_abi_version() == 103
    assert L.tdp_status_str(4) == b"capacity exceeded"
    assert L.tdp_filter_workspace(0) >= 0
    assert L.tdp_join_default_slots(3_000_000) == 1 << 23
    assert L.tdp_join_default_slots(0) == 8 and L.tdp_join_default_slots(5) == 16
    old = L.tdp_set_spin_limit(1000)
    assert L.tdp_set_spin_limit(old) == 1000


def test_host_argument_errors_without_launch():
    """Invalid arguments are rejected on the host before any launch."""
    import ctypes as C
    L = _lib.lib()
    # negative row count
    st = L.tdp_filter(None, 0, None, 0, -1, None, None, 0, C.c_void_p(8), None, 0, None, None, 0, None, None)
    assert st == 1
    # bad top-k k
    st = L.tdp_topk(None, None, 0, None, 0, C.c_void_p(8), C.c_void_p(8), None, None, 0, None, None)
    assert st == 1
    # soft op with tau <= 0
    st = L.tdp_soft_filter_fwd(None, None, None, 0.0, 0, None, None)
    assert st == 1
    # group-join: an empty key range, and its workspace query
    assert L.tdp_groupjoin_workspace(10, 5, 4, 1, 0) == 0
    assert L.tdp_groupjoin_workspace(10, 1, 15_000_000, 1, 0) > 15_000_000 // 32 * 12
    assert L.tdp_groupjoin_workspace(10, 1, 100, 1, 17) == 0  # top-k of at most 16
    st = L.tdp_groupjoin(None, 0, None, 0, 0, None, 0, None, 0, None, 0, 0, None, 0, 5, 4, None, 0, None, None, 0,
                         None, None, 0, 0, None, None, None, None, 0, None, None)
    assert st == 1
