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


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program gcc compiles
    against include/exactmap.h."""
    import subprocess
    import tempfile
    body = "\n".join(f'    printf("%s %zu\\n", "{f}", offsetof({struct}, {f}));' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"exactmap.h\"\nint main(void) {\n"
           f'    printf("sizeof %zu\\n", sizeof({struct}));\n{body}\n    return 0;\n}}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_struct_layouts_match_header():
    """The ctypes mirrors of em_params and em_snapshot have the header's
    size and field offsets."""
    from paper_2410_15227_gb300 import _native
    for cls, name in ((_native.EmParams, "em_params"), (_native.EmSnapshot, "em_snapshot")):
        fields = [f for f, _ in cls._fields_]
        lay = _c_layout(name, fields)
        assert lay["sizeof"] == ctypes.sizeof(cls), name
        for f in fields:
            assert lay[f] == getattr(cls, f).offset, (name, f)


def test_python_defaults_match_library():
    """api.Params() carries the values em_params_default() fills."""
    from dataclasses import fields
    from paper_2410_15227_gb300 import _native, api
    c = _native.EmParams()
    _native.lib().em_params_default(ctypes.byref(c))
    p = api.Params()
    for f in fields(p):
        assert getattr(c, f.name) == getattr(p, f.name), f.name


def test_batch_handle_argument_checks():
    """map_batch_create / add / get / destroy reject bad arguments with
    EM_EINVAL without touching a GPU."""
    import ctypes as C
    from paper_2410_15227_gb300 import _native
    L = _native.lib()
    p = _native.EmParams()
    L.em_params_default(C.byref(p))
    h = C.c_void_p()
    assert L.map_batch_create(-1, C.byref(p), 4, C.byref(h)) == _native.EM_EINVAL
    assert L.map_batch_create(0, C.byref(p), 0, C.byref(h)) == _native.EM_EINVAL
    assert L.map_batch_create(0, None, 4, C.byref(h)) == _native.EM_EINVAL
    assert L.map_batch_create(0, C.byref(p), 4, C.byref(h)) == _native.EM_OK
    rec = _native.EmSnapshot()   # all NULL: an invalid record
    assert L.map_batch_add(h, C.byref(rec), None) == _native.EM_EINVAL
    assert L.map_batch_get(h, 0, C.byref(rec)) == _native.EM_EINVAL   # nothing added
    assert L.map_batch_run(None, 0, None, None, None) == _native.EM_EINVAL
    assert L.map_batch_destroy(h) == _native.EM_OK
    assert L.map_batch_destroy(None) == _native.EM_OK
