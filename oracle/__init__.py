"""CPU oracle for certified-split lexing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import this package.  The GPU library never
loads it and shares no code with it.

The arithmetic lives in ``lexoracle.c`` (plain C, compiled with gcc on first
use); this module marshals numpy arrays through ctypes and adds the chunked
reference run used by the tests:

* ``lex``            -- the longest-match scanner of Section 3 (tok(w), con(w)).
* ``discard``        -- pi_I of Section 5.
* ``certificates``   -- Definitions 1-3, Corollary 2, Proposition 2.
* ``lex_chunks``     -- ordered concatenation of chunk-local scans, the right-hand
                        side of Theorems 1 and 3.
* ``plan``           -- the planner of Section 6: slide each of k-1 equal-division
                        targets forward to the next useful certified byte.
* ``par_lex``        -- not an oracle: the paper's method on host threads
                        (``parsplit.c``: the planner, one thread per chunk,
                        ordered concatenation), timed as the CPU baseline.
* ``contexts``       -- (submodule) entry contexts of the serial scan, their
                        candidate sets and chunk runs entered in a context:
                        splitting a token set with no certified byte.
* ``live``           -- (submodule) the live sets behind the failed-lookahead
                        guard and the guarded serial scan.
* ``windows``        -- (submodule) certified two-byte split windows.
* ``model``          -- (submodule) FP64 reference of the entry-context model.

Parity pins: tests/test_oracle_pins.py (worked examples of the paper),
tests/test_oracle_contexts.py (exhaustive checks of the entry contexts),
tests/test_oracle_bruteforce.py (exhaustive checks on tiny token sets),
tests/test_oracle_re.py (Python ``re.fullmatch`` cross-check of the scanner),
tests/test_oracle_discard_plan.py (hand-written pi_I streams and plans),
tests/test_oracle_live.py, tests/test_oracle_windows.py, tests/test_oracle_model.py.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lexoracle.c")
_SRC_PAR = os.path.join(_HERE, "parsplit.c")
CFLAGS = ["-O2", "-std=c11", "-pthread"]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblexoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lexoracle.c into oracle/_build/liblexoracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in (_SRC, _SRC_PAR))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-shared", "-fPIC", _SRC, _SRC_PAR, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declare the C signatures on a loaded liblexoracle (also used by the
    mutation tests, which load deliberately broken copies)."""
    i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.orc_lex.restype = i64
    lib.orc_lex.argtypes = [i32, i32, p, p, p, i64, p, p, i64, p]
    lib.orc_filter.restype = i64
    lib.orc_filter.argtypes = [p, p, i64, p, i32, p, p]
    lib.orc_certificates.restype = ctypes.c_int
    lib.orc_certificates.argtypes = [i32, i32, p, p, p, i32, p, p, p, p, p, p]
    lib.par_lex.restype = i64
    lib.par_lex.argtypes = [i32, p, p, p, p, i32, p, i64, i32, p, p, i64, p, p, p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Automaton:
    """Full-table view of a compiled token set: delta[q, b] and tau[q]."""

    def __init__(self, dfa):
        self.n_states = int(dfa.n_states)
        self.q0 = int(dfa.q0)
        self.delta = np.ascontiguousarray(dfa.delta_full(), dtype=np.int32)
        self.tau = np.ascontiguousarray(dfa.accept, dtype=np.int32)
        self.n_kinds = int(max(dfa.n_kinds, int(self.tau.max()) + 1 if self.n_states else 0))


def _as_automaton(dfa) -> Automaton:
    return dfa if isinstance(dfa, Automaton) else Automaton(dfa)


def _as_bytes(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    return np.ascontiguousarray(data, dtype=np.uint8)


def lex(dfa, data, cap: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray, int]:
    """tok(w) and con(w) of the serial scan (Section 3).

    Returns (kinds int32[T], lens int64[T], con)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    lib = _load()
    n = int(w.size)
    cap = n if cap is None else int(cap)
    kinds = np.empty(max(cap, 1), dtype=np.int32)
    lens = np.empty(max(cap, 1), dtype=np.int64)
    con = ctypes.c_int64(0)
    wbuf = w if n else np.zeros(1, np.uint8)
    t = lib.orc_lex(a.n_states, a.q0, _ptr(a.delta), _ptr(a.tau), _ptr(wbuf), n, _ptr(kinds),
                    _ptr(lens), cap, ctypes.addressof(con))
    if t > cap:
        raise ValueError(f"token capacity {cap} too small for {t} tokens")
    return kinds[:t].copy(), lens[:t].copy(), int(con.value)


def discard(kinds: np.ndarray, lens: np.ndarray, discarded: Iterable[int], n_kinds: int
            ) -> Tuple[np.ndarray, np.ndarray]:
    """pi_I: delete every (kind, length) pair whose kind is discarded."""
    lib = _load()
    k = np.ascontiguousarray(kinds, dtype=np.int32)
    l = np.ascontiguousarray(lens, dtype=np.int64)
    in_I = np.zeros(max(n_kinds, 1), dtype=np.uint8)
    for d in discarded:
        in_I[int(d)] = 1
    ok = np.empty(max(k.size, 1), np.int32)
    ol = np.empty(max(k.size, 1), np.int64)
    kb = k if k.size else np.zeros(1, np.int32)
    lb = l if l.size else np.zeros(1, np.int64)
    m = lib.orc_filter(_ptr(kb), _ptr(lb), int(k.size), _ptr(in_I), int(n_kinds), _ptr(ok), _ptr(ol))
    return ok[:m].copy(), ol[:m].copy()


class Certificates:
    def __init__(self, exact_raw, modulo_raw, exact, modulo, live, reentrant):
        self.exact_raw = exact_raw
        self.modulo_raw = modulo_raw
        self.exact = exact          # useful exact set (Corollary 2)
        self.modulo = modulo        # useful modulo-I set (Proposition 2)
        self.live = live
        self.reentrant = reentrant

    @staticmethod
    def _set(mask) -> List[int]:
        return [b for b in range(256) if mask[b]]

    def exact_bytes(self) -> List[int]:
        return self._set(self.exact)

    def modulo_bytes(self) -> List[int]:
        return self._set(self.modulo)


def certificates(dfa, discarded: Sequence[int] = ()) -> Certificates:
    """Exact and modulo-I certificates of Definitions 2 and 3 (useful and raw)."""
    a = _as_automaton(dfa)
    lib = _load()
    in_I = np.zeros(max(a.n_kinds, 1), dtype=np.uint8)
    for d in discarded:
        in_I[int(d)] = 1
    er, mr, eu, mu = (np.zeros(256, np.uint8) for _ in range(4))
    live = np.zeros(max(a.n_states, 1), np.uint8)
    reent = ctypes.c_int32(0)
    rc = lib.orc_certificates(a.n_states, a.q0, _ptr(a.delta), _ptr(a.tau), _ptr(in_I), a.n_kinds,
                              _ptr(er), _ptr(mr), _ptr(eu), _ptr(mu), _ptr(live),
                              ctypes.addressof(reent))
    if rc != 0:
        raise ValueError("invalid automaton")
    return Certificates(er.astype(bool), mr.astype(bool), eu.astype(bool), mu.astype(bool),
                        live[:a.n_states].astype(bool), bool(reent.value))


def lex_chunks(dfa, data, cuts: Sequence[int]) -> Tuple[np.ndarray, np.ndarray, int]:
    """Concatenate chunk-local scans of w[c_j, c_{j+1}) (Theorems 1 and 3).

    ``cuts`` are the interior offsets.  Chunks are scanned in order; the first
    chunk that does not consume its whole slice ends the run, and its halting
    offset is reported as the consumed length (Corollary 1)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    bounds = [0] + sorted(int(c) for c in cuts) + [int(w.size)]
    ks: List[np.ndarray] = []
    ls: List[np.ndarray] = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        k, l, con = lex(a, w[lo:hi])
        ks.append(k)
        ls.append(l)
        if con < hi - lo:
            return (np.concatenate(ks) if ks else np.zeros(0, np.int32),
                    np.concatenate(ls) if ls else np.zeros(0, np.int64), lo + con)
    return (np.concatenate(ks) if ks else np.zeros(0, np.int32),
            np.concatenate(ls) if ls else np.zeros(0, np.int64), int(w.size))


def plan(data, useful: np.ndarray, k: int) -> List[int]:
    """Section 6 planner: for each of the k-1 equal-division targets, slide
    forward to the next byte in the useful certified set; a single chunk when
    the set is empty.  Returns the distinct interior cut offsets."""
    w = _as_bytes(data)
    n = int(w.size)
    if k <= 1 or n == 0 or not np.any(useful):
        return []
    is_cert = np.asarray(useful, dtype=bool)[w]
    cuts: List[int] = []
    for i in range(1, k):
        t = (n * i) // k
        while t < n and not is_cert[t]:
            t += 1
        if 0 < t < n and (not cuts or cuts[-1] < t):
            cuts.append(t)
    return cuts


def par_lex(dfa, data, useful: np.ndarray, discarded: Iterable[int] = (), k: int = 1,
            cap: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray, int, int, float]:
    """The paper's CPU method (``parsplit.c``): plan k chunks at useful
    certified bytes, scan each on its own thread (pi_I fused for a non-empty
    ``discarded``), concatenate in order.  Returns (kinds u16, lens u32, con,
    chunks, seconds from planning to the end of the concatenation)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    lib = _load()
    n = int(w.size)
    cap = n if cap is None else int(cap)
    ok = np.empty(max(cap, 1), np.uint16)
    ol = np.empty(max(cap, 1), np.uint32)
    use = np.ascontiguousarray(np.asarray(useful, dtype=bool).astype(np.uint8))
    I = list(discarded)
    in_I = np.zeros(max(a.n_kinds, 1), np.uint8)
    for d in I:
        in_I[int(d)] = 1
    con = ctypes.c_int64(0)
    chunks = ctypes.c_int32(0)
    sec = ctypes.c_double(0.0)
    wbuf = w if n else np.zeros(1, np.uint8)
    t = lib.par_lex(a.q0, _ptr(a.delta), _ptr(a.tau), _ptr(use), _ptr(in_I) if I else None, a.n_kinds,
                    _ptr(wbuf), n, int(k), _ptr(ok), _ptr(ol), cap, ctypes.addressof(con),
                    ctypes.addressof(chunks), ctypes.addressof(sec))
    if t < 0:
        raise MemoryError("par_lex: out of memory")
    if t > cap:
        raise ValueError(f"token capacity {cap} too small for {t} tokens")
    return ok[:t].copy(), ol[:t].copy(), int(con.value), int(chunks.value), float(sec.value)
