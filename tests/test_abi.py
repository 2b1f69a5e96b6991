"""The C-ABI library loads and exports what include/marchenko.h declares (no GPU)."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "marchenko.h")


def _lib():
    from paper_2106_04649_gb300 import _native as N
    if not os.path.exists(N.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc unavailable: cannot build libmarchenko.so")
        from paper_2106_04649_gb300 import build
        build.build()
    return N.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mk_[a-z_A-Z0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mk_plan", "mk_load_R", "mk_set_Gd_window", "mk_iterate", "mk_fetch_fields",
                     "mk_destroy", "mk_last_error", "mk_workspace_size", "mk_get_stats"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_desc_layout_matches_c():
    from paper_2106_04649_gb300 import _native as N
    # int32 x4, double x3, int32, uint32, int32 x2 -> 56 bytes with natural alignment
    assert ctypes.sizeof(N.MkDesc) == 56
    assert ctypes.sizeof(N.MkStats) == 64
    assert ctypes.sizeof(N.MkTuning) == 24


def test_workspace_size_and_validation_without_gpu():
    _lib()
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300 import binding as B
    from paper_2106_04649_gb300.api import Desc
    d = Desc(601, 601, 2048, 1, 0.004, 10.0, 60.0)
    assert d.nw == 492
    n = B.mk_workspace_size([d])
    r_bytes = 492 * 601 * 608 * 8
    assert r_bytes < n < r_bytes + 80 * 2**20
    assert B.mk_workspace_size([d, d]) == 2 * n
    bad = [Desc(601, 600, 2048, 1, 0.004, 10.0), Desc(10, 10, 1000, 1, 0.004, 10.0),
           Desc(10, 10, 64, 0, 0.004, 10.0), Desc(10, 10, 64, 1, 0.0, 10.0),
           Desc(10, 10, 64, 1, 0.004, 10.0, rprec=7),
           Desc(10, 10, 64, 1, 0.004, 10.0, rprec=4, flags=N.MK_FLAG_STREAM_R)]
    codes = []
    for b in bad:
        with pytest.raises(B.MarchenkoError) as ei:
            B.mk_workspace_size([b])
        codes.append(ei.value.status)
        assert B.mk_last_error(None)
    assert codes == [N.MK_ERR_UNSUPPORTED, N.MK_ERR_UNSUPPORTED, N.MK_ERR_ARG, N.MK_ERR_ARG,
                     N.MK_ERR_UNSUPPORTED, N.MK_ERR_UNSUPPORTED]
    # streaming R keeps only two frequency chunks on the device
    ds = Desc(601, 601, 2048, 1, 0.004, 10.0, 60.0, flags=N.MK_FLAG_STREAM_R)
    assert B.mk_workspace_size([ds]) < n - r_bytes // 2


def test_null_arguments_rejected_without_gpu():
    lib = _lib()
    from paper_2106_04649_gb300 import _native as N
    assert lib.mk_workspace_size(None, 1, None) == N.MK_ERR_ARG
    assert lib.mk_plan(None, 1, None, None, 0, None) == N.MK_ERR_ARG
    assert lib.mk_iterate(None, 1, None) == N.MK_ERR_ARG
    assert lib.mk_load_R(None, 0, None, 0, 0, 0) == N.MK_ERR_ARG
    assert lib.mk_destroy(None) == N.MK_OK
    assert b"null" in lib.mk_last_error(None)


def test_python_constants_match_header():
    """Every MK_ constant the binding defines has the header's value."""
    from paper_2106_04649_gb300 import _native as N
    text = open(HEADER).read()
    values = {}
    for name, expr in re.findall(r"#define\s+(MK_[A-Z0-9_]+)\s+\(?([^/\n]+?)\)?\s*(?:/\*|\n)", text):
        expr = expr.replace("u <<", " <<").replace("u)", ")").replace("0xFFu", "0xFF").strip().rstrip("u")
        try:
            values[name] = eval(expr, {"size_t": int})
        except Exception:
            pass
    for name, val in re.findall(r"\b(MK_(?:R|OK|ERR)_?[A-Z0-9_]*)\s*=\s*(\d+)", text):
        values[name] = int(val)
    checked = 0
    for name, val in values.items():
        if hasattr(N, name):
            assert getattr(N, name) == val, name
            checked += 1
    assert checked >= 20
