"""Seeded synthetic corpora (Python front end of ``corpus.c``).

Workloads (sizes and seeds fixed so that every run sees the same bytes):

=================  ==========================  ==============  ===========
name               generator                   default size    seed
=================  ==========================  ==============  ===========
arith              arith token stream          1 MiB           0x1EC50001
json               newline-delimited JSON      512 MiB         0x1EC50002
clike              C-like statement lines      512 MiB         0x1EC50003
clike_block        C-like + block comments     512 MiB         0x1EC50005
=================  ==========================  ==============  ===========
"""

from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corpus.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libcorpus.so")
_lock = threading.Lock()
_lib = None

MiB = 1 << 20

WORKLOADS = {
    "arith": ("gen_arith", 1 * MiB, 0x1EC50001),
    "json": ("gen_json", 512 * MiB, 0x1EC50002),
    "clike": ("gen_clike", 512 * MiB, 0x1EC50003),
    "clike_block": ("gen_clike_block", 512 * MiB, 0x1EC50005),
}


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for fn in ("gen_arith", "gen_json", "gen_clike", "gen_clike_block"):
                f = getattr(lib, fn)
                f.restype = ctypes.c_uint64
                f.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64]
            _lib = lib
    return _lib


def generate(name: str, n: int | None = None, seed: int | None = None,
             out: np.ndarray | None = None) -> np.ndarray:
    """Generate workload ``name`` with exactly ``n`` bytes (default size and
    seed from the table above).  ``out`` may supply a uint8 buffer (e.g. the
    numpy view of pinned host memory)."""
    fn, n_def, seed_def = WORKLOADS[name]
    n = n_def if n is None else int(n)
    seed = seed_def if seed is None else int(seed)
    buf = np.empty(max(n, 1), dtype=np.uint8) if out is None else out
    assert buf.dtype == np.uint8 and buf.size >= n and buf.flags.c_contiguous
    if n:
        got = getattr(_load(), fn)(seed, buf.ctypes.data, n)
        assert got == n
    return buf[:n]


def sha256(buf: np.ndarray) -> str:
    return hashlib.sha256(memoryview(np.ascontiguousarray(buf))).hexdigest()
