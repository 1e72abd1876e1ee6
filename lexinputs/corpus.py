"""Seeded synthetic corpora (Python front end of ``corpus.c``).

Workloads (sizes and seeds fixed so that every run sees the same bytes):

=================  ==========================  ==============  ===========
name               generator                   default size    seed
=================  ==========================  ==============  ===========
arith              arith token stream          1 MiB           0x1EC50001
json               newline-delimited JSON      512 MiB         0x1EC50002
clike              C-like statement lines      512 MiB         0x1EC50003
clike_block        C-like + block comments     512 MiB         0x1EC50005
clike_block_framed the same, 0x1E before every  512 MiB         0x1EC50006
                   line or comment (producer
                   framing, Section 7.1)
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
    "clike_block_framed": ("gen_clike_block_framed", 512 * MiB, 0x1EC50006),
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
            for fn in ("gen_arith", "gen_json", "gen_clike", "gen_clike_block", "gen_clike_block_framed"):
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


# ---------------------------------------------------------------------------
# Document batches: many documents of mixed token sets (the batched launch)
# ---------------------------------------------------------------------------
BATCH_SEED = 0x1EC50004


def _splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def batch_spec(n_docs: int = 4096, seed: int = BATCH_SEED, median: int = 128 << 10, sigma: float = 1.66,
               lo: int = 1 << 10, hi: int = 16 << 20, names=("json", "clike")):
    """(name, size, seed) of each document: sizes lognormal (median, sigma)
    clamped to [lo, hi], the workload drawn uniformly from ``names``; every
    draw comes from a splitmix64 stream, so the batch is the same on any
    machine."""
    import math
    state = seed
    out = []
    for i in range(n_docs):
        state = _splitmix64(state)
        u1 = ((state >> 11) + 1) / float(1 << 53)          # (0, 1]
        state = _splitmix64(state)
        u2 = (state >> 11) / float(1 << 53)                # [0, 1)
        state = _splitmix64(state)
        which = names[state % len(names)]
        z = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
        size = int(round(median * math.exp(sigma * z)))
        size = min(max(size, lo), hi)
        out.append((which, size, (seed << 16) ^ (i + 1)))
    return out


def generate_batch(spec, align: int = 16):
    """Generate every document of ``spec`` into one buffer; returns (buffer,
    offsets).  Document i occupies buffer[offsets[i] : offsets[i] + size_i];
    offsets are multiples of ``align``."""
    offs, pos = [], 0
    for _, size, _ in spec:
        offs.append(pos)
        pos += (size + align - 1) // align * align
    buf = np.zeros(max(pos, 1), dtype=np.uint8)
    for (name, size, s), o in zip(spec, offs):
        if size:
            generate(name, size, seed=s, out=buf[o:o + size])
    return buf, offs
