"""The C-ABI library builds, loads and exports every symbol include/hodlr.h
declares; argument validation runs before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    from paper_2407_21637_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hodlr_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"hodlr_import", "hodlr_matvec", "hodlr_destroy"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_bindings_cover_the_header(lib):
    from paper_2407_21637_gb300 import _lib
    assert declared_functions() == set(_lib.SIGNATURES)


def test_status_strings(lib):
    for s in range(8):
        assert lib.hodlr_status_string(s)
    assert lib.hodlr_status_string(99) == b"unknown status"


def test_validation_before_device_work(lib):
    from paper_2407_21637_gb300 import _lib
    h = ctypes.c_void_p()
    opts = _lib.Opts(eps=1e-6, work=1, tier_mask=0b11111, per_block=0, max_nrhs=0)
    D = (ctypes.POINTER(ctypes.c_double) * 1)()
    # null opts
    assert lib.hodlr_import(16, 0, None, None, None, D, None, None, ctypes.byref(h)) == 1
    # 2^depth > n
    assert lib.hodlr_import(4, 3, None, None, None, D, ctypes.byref(opts), None, ctypes.byref(h)) == 1
    # bad working precision
    bad = _lib.Opts(eps=1e-6, work=3, tier_mask=1, per_block=0, max_nrhs=0)
    assert lib.hodlr_import(16, 0, None, None, None, D, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"working precision" in lib.hodlr_last_error()
    # eps out of range
    bad = _lib.Opts(eps=1.5, work=1, tier_mask=1, per_block=0, max_nrhs=0)
    assert lib.hodlr_import(16, 0, None, None, None, D, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    # unknown tier bits
    bad = _lib.Opts(eps=1e-3, work=1, tier_mask=1 << 9, per_block=0, max_nrhs=0)
    assert lib.hodlr_import(16, 0, None, None, None, D, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    # matvec on a null handle, dense checker with a bad kernel kind
    assert lib.hodlr_matvec(None, 1, None, 1, None, 1, 1, None) == 1
    assert lib.hodlr_dense_kernel_matvec(8, 2, ctypes.c_void_p(8), 3, 0.0, 1.0, 0.0, 8, None, 1,
                                         ctypes.c_void_p(8), 1, ctypes.c_void_p(8), 1, None) == 1
    assert h.value is None
    lib.hodlr_destroy(None)
    # partitioned product: null handle / part
    part = ctypes.c_void_p()
    assert lib.hodlr_part_create(None, 0, 0, 1, ctypes.byref(part)) == 1
    assert part.value is None
    assert lib.hodlr_part_partial(None, None, 1, None, None) == 1
    assert lib.hodlr_part_finish(None, None, 1, None, None, 1, None) == 1
    assert lib.hodlr_part_info(None, None, None, None) == 1
    lib.hodlr_part_destroy(None)


def test_load_rejects_bad_files_before_device_work(lib, tmp_path):
    h = ctypes.c_void_p()
    assert lib.hodlr_load(str(tmp_path / "missing.hodlr").encode(), None, ctypes.byref(h)) == 1
    bad = tmp_path / "bad.hodlr"
    bad.write_bytes(b"NOTHODLR" + bytes(64))
    assert lib.hodlr_load(str(bad).encode(), None, ctypes.byref(h)) == 1
    assert b"magic" in lib.hodlr_last_error()
    short = tmp_path / "short.hodlr"
    short.write_bytes(b"HODLRSV1" + bytes(8))
    assert lib.hodlr_load(str(short).encode(), None, ctypes.byref(h)) == 1
    assert not h.value
