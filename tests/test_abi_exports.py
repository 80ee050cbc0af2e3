"""The engine library loads without a GPU and exports every entry point that
include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lob_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2308_13289_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lob_create", "lob_process_batch", "lob_inject_orders", "lob_get_levels",
                 "lob_get_trades", "lob_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), "liblob.so does not export %s" % name


def test_binding_covers_every_declared_symbol():
    from paper_2308_13289_b300 import _abi
    missing = declared_functions() - set(_abi.SIGNATURES)
    assert not missing, missing


def test_cpu_only_calls_fail_cleanly(lib):
    lib.lob_abi_version.restype = ctypes.c_int
    assert lib.lob_abi_version() == 2
    lib.lob_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lob_destroy(None) == 0
    lib.lob_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.lob_create(None, None, None) == -1
    lib.lob_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.lob_last_error()
    # argument errors are caught on the host before any launch
    lib.lob_get_levels_books.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int32] + [ctypes.c_void_p] * 5
    one = ctypes.c_void_p(16)
    assert lib.lob_get_levels_books(None, one, 1, 10, one, one, one, one, None) == -1
    assert b"lob_get_levels_books" in lib.lob_last_error()
    # the serving executor checks its descriptor and handles before any CUDA call
    lib.lob_serve_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.lob_serve_create(ctypes.byref(out), None) == -1
    from paper_2308_13289_b300._abi import LobServeDesc
    desc = LobServeDesc(slots=4, max_msgs=10, depth=10, ring=8)  # null pointers
    assert lib.lob_serve_create(ctypes.byref(out), ctypes.byref(desc)) == -1
    assert b"invalid descriptor" in lib.lob_last_error() and not out.value
    lib.lob_serve_tick.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + \
        [ctypes.c_void_p] * 5
    assert lib.lob_serve_tick(None, 0, 0, None, None, None, None, None) == -1
    lib.lob_serve_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lob_serve_destroy(None) == 0
