"""The C-ABI library builds, loads, and exports every function that
include/*.h declares (no GPU needed; no compute calls)."""

from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(cht_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2011_11762_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("cht_mat_from_blocks", "cht_symbolic_multiply", "cht_multiply",
                     "cht_multiply_backward", "cht_to_dense"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_build_exports_every_declared_symbol():
    # the bounds-checked debug variant (-DCHT_BOUNDS_CHECK) builds from the
    # same sources and exports the same boundary
    from paper_2011_11762_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libcht_checked.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2011_11762_gb300 import _lib
    assert _declared_functions() <= set(_lib.SIGNATURES)


def test_host_only_calls(libpath):
    import paper_2011_11762_gb300 as cht
    lib = cht.load()
    assert lib.cht_status_str(cht.CHT_ERR_TIMEOUT) == b"CHT_ERR_TIMEOUT"
    assert lib.cht_status_str(0) == b"CHT_OK"
    assert lib.cht_set_option(cht.OPT_SCHEDULE, 7) == cht.CHT_ERR_INVALID
    assert b"invalid option" in lib.cht_last_error()
    v = ctypes.c_int64()
    assert lib.cht_get_option(cht.OPT_WAIT_BUDGET_NS, ctypes.byref(v)) == 0
    assert v.value == 2_000_000_000
    # argument checks happen on the host before any device work
    h = ctypes.c_void_p()
    assert lib.cht_mat_from_blocks(100, 32, 0, None, None, None, None,
                                   ctypes.byref(h)) == cht.CHT_ERR_INVALID
    assert lib.cht_mat_from_blocks(128, 16, 0, None, None, None, None,
                                   ctypes.byref(h)) == cht.CHT_ERR_INVALID
    assert lib.cht_multiply(None, None, None, 0, 0, None, None, None) == cht.CHT_ERR_INVALID
    assert lib.cht_set_allocator(ctypes.c_void_p(1), None, None) == cht.CHT_ERR_INVALID
    assert lib.cht_batch_create(0, None, None, None, 0, 0, None,
                                ctypes.byref(h)) == cht.CHT_ERR_INVALID
    # the operations around the product check their arguments on the host too
    n = ctypes.c_int64()
    d = ctypes.c_double()
    inv = cht.CHT_ERR_INVALID
    assert lib.cht_symbolic_multiply_spamm(None, None, -1.0, None, ctypes.byref(h),
                                           None, None) == inv
    assert lib.cht_symbolic_multiply_symsquare(None, None, ctypes.byref(h), ctypes.byref(n),
                                               ctypes.byref(n)) == inv
    assert lib.cht_symbolic_multiply_upper(None, None, None, ctypes.byref(h), None, None) == inv
    assert lib.cht_mat_mirror_upper(None, None, ctypes.byref(h)) == inv
    assert lib.cht_add(1.0, None, 1.0, None, None, ctypes.byref(h)) == inv
    assert lib.cht_add_identity(1.0, None, 1.0, None, ctypes.byref(h)) == inv
    assert lib.cht_truncate(None, 1e-6, cht.CHT_TRUNC_FRO, None, ctypes.byref(h),
                            ctypes.byref(d)) == inv
    assert lib.cht_multiply_to_host(None, None, None, None, None, 0) == inv
    assert b"nchunks" in lib.cht_last_error()
    # shape limits of the boundary: leaf size 32..64 in steps of 8, n a
    # multiple of b, a leaf count that fits int32, 16-byte aligned values, and
    # at most 2^21 leaves per grid side (the 64-bit Morton pair keys)
    for n, b, nb in ((4096, 16, 0), (4096, 72, 0), (4096, 36, 0), (4000, 64, 0),
                     (4096, 64, -1), (4096, 64, 1 << 31), (0, 64, 0), (-64, 64, 0)):
        assert lib.cht_mat_from_blocks(n, b, nb, None, None, None, None,
                                       ctypes.byref(h)) == inv, (n, b, nb)
    dummy = ctypes.c_void_p(64)
    assert lib.cht_mat_from_blocks(4096, 64, 1, dummy, dummy, ctypes.c_void_p(72), None,
                                   ctypes.byref(h)) == inv
    assert b"aligned" in lib.cht_last_error()
    assert lib.cht_mat_from_blocks(64 * ((1 << 21) + 1), 64, 0, None, None, None, None,
                                   ctypes.byref(h)) == cht.CHT_ERR_UNSUPPORTED
    assert b"2^21" in lib.cht_last_error()
    for code in (cht.CHT_ERR_INVALID, cht.CHT_ERR_SHAPE, cht.CHT_ERR_DUPLICATE,
                 cht.CHT_ERR_OOM, cht.CHT_ERR_CUDA, cht.CHT_ERR_UNSUPPORTED):
        assert lib.cht_status_str(code).startswith(b"CHT_ERR_")


def test_product_path_has_no_oracle_dependency():
    # the GPU library and its binding never import or link the oracle
    pkg = os.path.join(ROOT, "paper_2011_11762_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isdir(path) or "_build" in path:
            continue
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "liborc" not in text, path
