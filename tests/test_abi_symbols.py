"""The C-ABI library loads without a GPU and exports every function include/bras.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2607_12138_b300", "libbras.so")
HEADER = os.path.join(ROOT, "include", "bras.h")


def _declared():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(bras_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_header_symbols():
    if not os.path.exists(LIB):
        from paper_2607_12138_b300 import build
        build.build()
    lib = ctypes.CDLL(LIB)
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    lib = ctypes.CDLL(LIB)
    lib.bras_n_local.restype = ctypes.c_int
    nl = lambda d, s, k, b=0: lib.bras_n_local(d, s, k, b)
    assert [nl(3, 0, p) for p in (1, 2, 3, 4)] == [4, 10, 20, 35]
    assert [nl(2, 0, p) for p in (1, 2, 3, 4)] == [3, 6, 10, 15]
    assert [nl(3, 0, p, 1) for p in (1, 2, 3, 4)] == [4, 10, 20, 35]          # Bernstein
    assert [nl(3, 1, k) for k in (1, 2, 3, 4)] == [6, 20, 45, 84]
    assert [nl(3, 2, k) for k in (1, 2, 3, 4)] == [4, 15, 36, 70]
    assert [nl(2, 1, k) for k in (1, 2, 3, 4)] == [3, 8, 15, 24]
    assert [nl(2, 2, k) for k in (1, 2, 3, 4)] == [3, 8, 15, 24]
    for s in (1, 2):                                                             # N2curl, BDM
        assert [nl(3, s, k, 1) for k in (1, 2, 3, 4)] == [12, 30, 60, 105]
        assert [nl(2, s, k, 1) for k in (1, 2, 3, 4)] == [6, 12, 20, 30]
        assert nl(3, s, 5, 1) == -1
    assert nl(2, 1, 5) == -1 and nl(3, 2, 5) == -1 and nl(3, 0, 5) == -1
    lib.bras_status_string.restype = ctypes.c_char_p
    assert lib.bras_status_string(-5) == b"local mass matrix not SPD"
    assert lib.bras_status_string(-11) == b"a kernel's bounded wait ran out"
    out = ctypes.c_void_p(1)
    # invalid arguments are rejected before any device work
    assert lib.bras_setup(ctypes.byref(out), 4, 0, 1, 0, None, 0, None, 0, None, None, None, None, None) == -1
    assert out.value is None
