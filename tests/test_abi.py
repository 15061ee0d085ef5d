"""The C-ABI library builds, loads and exports every function include/rt.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os

from paper_2303_11103_gb300 import build, rt


def test_header_symbols_exported():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = rt.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/rt.h but not exported"


def test_binding_covers_header():
    L = rt.lib()
    for n in rt.header_symbols():
        f = getattr(L, n)
        assert f.restype is ctypes.c_int, f"{n} has no binding"


def test_error_paths_without_gpu():
    # rt_create must fail cleanly (no abort) when no device is visible / index invalid
    h = ctypes.c_void_p()
    code = rt.lib().rt_create(ctypes.byref(h), 10_000, None)
    assert code == -1 and not h.value
    assert rt.lib().rt_destroy(None) == 0
