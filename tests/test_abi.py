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
