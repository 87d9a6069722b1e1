"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point the header declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "deann_gb300.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kde_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_02736_gb300 import build
    path = build.build()
    import paper_2107_02736_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_path():
    names = _declared()
    for want in ("kde_build", "kde_query", "kde_exact", "kde_query_rs", "kde_search",
                 "kde_grad", "kde_grad_with_neighbors", "kde_query_with_neighbors",
                 "kde_sample_indices", "kde_mean_shift",
                 "kde_export_ivf", "kde_free"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_covers_every_status(lib):
    for s in range(6):
        assert lib.kde_strerror(s)
    assert lib.kde_strerror(99) == b"unknown status"


def test_build_rejects_null_out_without_gpu(lib):
    X = (ctypes.c_float * 4)(1, 2, 3, 4)
    st = lib.kde_build(X, 2, 2, 0, 1.0, 1, 0, None, None)
    assert st == 1
    assert b"out" in lib.kde_last_error()


@pytest.mark.parametrize("n,d,h,kern,nlist,msg", [
    (0, 2, 1.0, 0, 1, b"n must"),
    (2, 0, 1.0, 0, 1, b"d must"),
    (2, 5000, 1.0, 0, 1, b"d must"),
    (2, 2, -1.0, 0, 1, b"h must"),
    (2, 2, float("inf"), 0, 1, b"h must"),
    (2, 2, 1.0, 7, 1, b"kernel"),
    (2, 2, 1.0, 0, 3, b"nlist"),
])
def test_build_argument_checks(lib, n, d, h, kern, nlist, msg):
    X = (ctypes.c_float * 4)(1, 2, 3, 4)
    out = ctypes.c_void_p()
    st = lib.kde_build(X, n, d, kern, h, nlist, 0, None, ctypes.byref(out))
    assert st == 1 and not out.value
    assert msg in lib.kde_last_error()


def test_calls_reject_null_index(lib):
    assert lib.kde_query(None, None, 0, 1, 1, 1, 0, None, None, None) == 1
    assert lib.kde_exact(None, None, 0, None, None) == 1
    assert lib.kde_set_bandwidth(None, 1.0) == 1
    assert lib.kde_set_scan_tile(None, 1, 64) == 1
    assert lib.kde_set_phase_window(None, 1 << 20) == 1
    lib.kde_free(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2107_02736_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg._build_mod, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        pkg.load_library()


@pytest.mark.parametrize("cname,pyname", [("kde_opts", "_Opts"), ("kde_profile", "_Profile")])
def test_structs_match_binding(tmp_path, cname, pyname):
    """The binding's ctypes mirror of a header struct has its fields, in order,
    at the same offsets and with the same size (compiled against the header)."""
    import paper_2107_02736_gb300 as pkg
    mirror = getattr(pkg, pyname)
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\} " + cname + ";", text).group(1)
    fields = re.findall(r"(\w+)\s*(?:\[\w+\])?\s*;", body)
    assert [f[0] for f in mirror._fields_] == fields
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "deann_gb300.h"\n'
                   f"int main(void) {{ printf(\"%zu\", sizeof({cname}));"
                   + "".join(f' printf(" %zu", offsetof({cname}, {f}));' for f in fields)
                   + " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(mirror)] + [getattr(mirror, f).offset for f in fields]
    assert got == want


def test_view_argument_errors_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.kde_index_view(None, ctypes.byref(out)) == 1
    assert b"NULL" in lib.kde_last_error()
    assert lib.kde_index_view(None, None) == 1
