"""Entry contexts for splitting without certified bytes -- TEST INFRASTRUCTURE ONLY.

For a token set whose certified sets are empty (the paper's refused sets),
the input is still split at arbitrary offsets p_0 = 0 < p_1 < ... and each
chunk is scanned from its *entry context*: the state of the serial scan of
Section 3 at its start.  Plain definitions, following the serial scan:

* context(p) = BOUNDARY when some serial token ends (or starts) at p, else
  delta*(q0, w[s, p)) for the serial token [s, e) with s < p < e.  Scanning
  on from that state finds the same token end e, because the longest match
  keeps the last accepting position and e > p.
* candidates(b) = {BOUNDARY} together with every delta(q, b) that lies in Q+:
  the context after byte b, whatever came before, is one of them (the
  candidate set of enumerative splitting).
* chunk_run(p0, p1, c): the tokens that start in [p0, p1) when the scan
  enters p0 in context c -- a token straddling p0 belongs to the previous
  chunk, one straddling p1 to this one -- and the context at p1.
* chained(starts): chunk runs from context(0) = BOUNDARY, each entering in
  the previous one's exit context; equal to tok(w) and con(w).

Pure-Python loops: for small inputs only.
"""

from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import Automaton, _as_automaton, _as_bytes, certificates, lex

BOUNDARY = -1


def contexts(dfa, data) -> List[Optional[int]]:
    """context(p) for p = 0 .. n (None past con(w), where the scan halted)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    n = int(w.size)
    kinds, lens, con = lex(a, w)
    ctx: List[Optional[int]] = [None] * (n + 1)
    s = 0
    for ln in lens.tolist():
        ctx[s] = BOUNDARY
        q = a.q0
        for p in range(s + 1, s + ln):
            q = int(a.delta[q, w[p - 1]])
            ctx[p] = q
        s += ln
    ctx[s] = BOUNDARY           # s == con(w)
    return ctx


def live_states(dfa) -> np.ndarray:
    """Q+ (reachable and co-accessible), from the certificate computation."""
    return certificates(dfa).live


def candidates(dfa, b: int, live: Optional[np.ndarray] = None) -> List[int]:
    """BOUNDARY first, then the distinct delta(q, b) in Q+ for q in Q+, ascending."""
    a = _as_automaton(dfa)
    live = live_states(a) if live is None else live
    out = set()
    for q in range(a.n_states):
        if live[q]:
            t = int(a.delta[q, b])
            if t >= 0 and live[t]:
                out.add(t)
    return [BOUNDARY] + sorted(out)


def _run(a: Automaton, w: np.ndarray, q: int, j: int) -> Tuple[Optional[int], int]:
    """From state q before byte j, follow delta while defined; the last
    accepting end position (> j) and its kind, or (None, -1)."""
    n = int(w.size)
    last, kind = None, -1
    while j < n:
        t = int(a.delta[q, w[j]])
        if t < 0:
            break
        q = t
        j += 1
        if a.tau[q] >= 0:
            last, kind = j, int(a.tau[q])
    return last, kind


def _state_after(a: Automaton, w: np.ndarray, q: int, lo: int, hi: int) -> int:
    for j in range(lo, hi):
        q = int(a.delta[q, w[j]])
    return q


def chunk_run(dfa, data, p0: int, p1: int, ctx: int):
    """(tokens, exit context, failure offset) of the chunk [p0, p1) entered in
    context ``ctx``.  tokens: list of (kind, length) of the tokens starting in
    [p0, p1); exit: context at p1 (None when the scan fails in the chunk);
    failure: the offset where no accepting prefix exists, or None.  A
    mid-token ``ctx`` from which no accepting position past p0 is reachable
    cannot be the true context; it returns (None, None, None)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    toks: List[Tuple[int, int]] = []
    pos = p0
    if ctx != BOUNDARY:
        e, _ = _run(a, w, ctx, p0)
        if e is None:
            return None, None, None
        if e >= p1:
            return toks, (BOUNDARY if e == p1 else _state_after(a, w, ctx, p0, p1)), None
        pos = e
    while pos < p1:
        e, kind = _run(a, w, a.q0, pos)
        if e is None:
            return toks, None, pos
        toks.append((kind, e - pos))
        if e >= p1:
            return toks, (BOUNDARY if e == p1 else _state_after(a, w, a.q0, pos, p1)), None
        pos = e
    return toks, BOUNDARY, None


def chained(dfa, data, starts: Sequence[int]):
    """Chunk runs in order from BOUNDARY at offset 0, each entered in the
    previous exit context: (kinds, lens, con)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    n = int(w.size)
    bounds = sorted(set([0] + [int(s) for s in starts if 0 < s < n])) + [n]
    ctx = BOUNDARY
    ks: List[int] = []
    ls: List[int] = []
    for p0, p1 in zip(bounds[:-1], bounds[1:]):
        toks, ctx, fail = chunk_run(a, w, p0, p1, ctx)
        assert toks is not None, "a chained entry context is always valid"
        ks += [k for k, _ in toks]
        ls += [l for _, l in toks]
        if fail is not None:
            return np.array(ks, np.int32), np.array(ls, np.int64), fail
    return np.array(ks, np.int32), np.array(ls, np.int64), n
