"""The C-ABI library loads and exports every function include/lexgpu.h declares."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lx_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lexlib):
    lib = ctypes.CDLL(lexlib.LIB_PATH)
    names = declared_functions()
    assert "lx_lex" in names and "lx_compile_tokenset" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(lexlib.EXPORTED) == names


def test_strerror(lexlib):
    assert lexlib.lx_strerror(0) == "ok"
    assert "capacity" in lexlib.lx_strerror(lexlib.LX_E_CAPACITY)


def test_argument_errors_before_any_gpu_work(lexlib):
    """Malformed calls are refused by the library's argument checks, which
    run before any CUDA call (so these need no GPU): a missing context or
    token set, a mode outside the three of Theorems 1 and 3, an input pointer
    missing for a non-empty input, output arrays missing for a non-zero
    capacity, and for lx_lex_noalloc an input beyond its fixed scratch."""
    from lexinputs import tokensets as T
    lg = lexlib
    lib = lg.load_library()
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    nt, con = ctypes.c_uint64(7), ctypes.c_uint64(7)
    out = ctypes.byref(nt), ctypes.byref(con)
    dummy = ctypes.create_string_buffer(64)          # never dereferenced on these paths
    p = ctypes.addressof(dummy)
    M = lg.LX_FILTERED_MODULO
    for fn in (lib.lx_lex, lib.lx_lex_host):
        assert fn(None, ts.handle, p, 16, M, p, p, 16, *out, None) == lg.LX_E_INVAL
        assert fn(p, None, p, 16, M, p, p, 16, *out, None) == lg.LX_E_INVAL
        assert fn(p, ts.handle, p, 16, 3, p, p, 16, *out, None) == lg.LX_E_MODE
        assert fn(p, ts.handle, p, 16, -1, p, p, 16, *out, None) == lg.LX_E_MODE
        assert fn(p, ts.handle, None, 16, M, p, p, 16, *out, None) == lg.LX_E_INVAL
        assert fn(p, ts.handle, p, 16, M, None, p, 16, *out, None) == lg.LX_E_INVAL
        assert fn(p, ts.handle, p, 16, M, p, None, 16, *out, None) == lg.LX_E_INVAL
        assert fn(p, ts.handle, p, 16, M, p, p, 16, None, ctypes.byref(con), None) == lg.LX_E_INVAL
    na = lib.lx_lex_noalloc
    assert na(None, p, 16, M, p, p, 16, *out, None) == lg.LX_E_INVAL
    assert na(ts.handle, p, 16, 5, p, p, 16, *out, None) == lg.LX_E_MODE
    assert na(ts.handle, None, 16, M, p, p, 16, *out, None) == lg.LX_E_INVAL
    assert na(ts.handle, p, lg.LX_NOALLOC_MAX_INPUT + 1, M, p, p, 16, *out, None) == lg.LX_E_INVAL
    assert na(ts.handle, p, 0, M, p, p, 16, *out, None) == lg.LX_OK    # empty input: no tokens
    assert nt.value == 0 and con.value == 0
