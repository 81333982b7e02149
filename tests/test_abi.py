"""The C-ABI library builds, loads and exports every entry point of include/diter.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(di_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6158_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared("diter.h")
    for must in ["di_graph_create", "di_solve", "di_query", "di_power", "di_free", "di_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared("diter.h"):
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_1202_6158_gb300 import _lib
    lib = _lib.load()
    for name in declared("diter.h"):
        assert getattr(lib, name).argtypes is not None or name in ("di_last_error", "di_version"), name


def test_version_and_error_without_gpu(lib):
    lib.di_version.restype = ctypes.c_char_p
    assert b"libditer" in lib.di_version()
    lib.di_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.di_last_error(), bytes)


def test_host_side_argument_checks_need_no_gpu(lib):
    """Arguments rejected before any CUDA call return DI_EINVAL with a message."""
    out = ctypes.c_void_p()
    lib.di_graph_create.restype = ctypes.c_int
    lib.di_graph_create.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    rp = (ctypes.c_int32 * 2)(0, 0)
    assert lib.di_graph_create(0, rp, None, 0, 0.85, None, None, ctypes.byref(out)) == 1
    assert lib.di_graph_create(1, rp, None, 0, 1.0, None, None, ctypes.byref(out)) == 1
    assert lib.di_graph_create(1, rp, None, 0, 0.0, None, None, ctypes.byref(out)) == 1
    assert lib.di_graph_create(1, None, None, 0, 0.5, None, None, ctypes.byref(out)) == 1
    assert out.value is None


@pytest.fixture(scope="module")
def dlib():
    from paper_1202_6158_gb300 import build
    return ctypes.CDLL(build.build(debug=True))


def test_debug_build_exports_the_same_boundary(dlib):
    """libditer_debug.so (DI_DEBUG: device-side index checks) has every entry point too."""
    for name in declared("diter.h"):
        assert hasattr(dlib, name), name


def test_debug_flag_tells_the_builds_apart(lib, dlib):
    lib.di_debug_build.restype = ctypes.c_int32
    dlib.di_debug_build.restype = ctypes.c_int32
    assert lib.di_debug_build() == 0 and dlib.di_debug_build() == 1
    # the release build refuses the self-test on the host, before any CUDA call
    w = ctypes.c_uint64(7)
    lib.di_debug_selftest.restype = ctypes.c_int
    assert lib.di_debug_selftest(ctypes.byref(w)) == 1 and w.value == 0
