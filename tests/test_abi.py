"""The C-ABI library builds, loads, and exports every symbol the header
declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "exactmap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char \*)\s*\*?\s*(\w+)\s*\(", src, re.M)))


def test_library_exports_header_symbols():
    from paper_2410_15227_gb300 import build, _native
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_native.SIGNATURES), set(names) ^ set(_native.SIGNATURES)


def test_binding_loads_and_reports_errors():
    from paper_2410_15227_gb300 import _native
    L = _native.lib()
    p = _native.EmParams()
    L.em_params_default(ctypes.byref(p))
    assert p.h_fact == 1.2 and p.leaf_max == 8 and p.precision == 0
    # a null context is rejected with EM_EINVAL and a message, without touching a GPU
    st = L.em_ctx_sync(None)
    assert st == _native.EM_EINVAL
    assert b"invalid argument" in L.em_last_error()
