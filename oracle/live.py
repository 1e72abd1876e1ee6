"""Liveness of scan states -- TEST INFRASTRUCTURE ONLY.

The failed-lookahead guard rests on one set per offset k of the input w:

    live_k = { q in Q+ : delta*(q, w[k..m)) is accepting for some m > k }

the states from which the longest-match scan of Section 3, standing before
byte k, still meets an accepting state.  A scan whose state is not in live_k
has already passed the last accepting position of its token (Section 9: the
quadratic pathology of failed lookahead, removed by tabulating the failed
(state, position) pairs, Reps, or by a right-to-left pass over the suffixes).

* ``live_sets``   -- the plain definition: from every state of Q+ at every
                     offset, follow delta over the input until it is
                     undefined; live iff an accepting state is met on the way.
* ``guarded_lex`` -- the serial scan of Section 3 that also ends a token as
                     soon as its state leaves live_k; returns the tokens and
                     the number of transitions it took (each token costs its
                     length plus at most one step).

Pure-Python loops over offsets (numpy over states): for small inputs only.
"""

from __future__ import annotations

from typing import Tuple

import numpy as np

from . import _as_automaton, _as_bytes, certificates


def live_sets(dfa, data) -> np.ndarray:
    """bool[n + 1, S]: row k is live_k (columns outside Q+ are False)."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    n = int(w.size)
    qplus = np.asarray(certificates(a).live, dtype=bool)
    acc = a.tau >= 0
    out = np.zeros((n + 1, a.n_states), dtype=bool)
    states = np.flatnonzero(qplus)
    for k in range(n + 1):
        cur = states.copy()            # one walker per start state
        start = states.copy()
        seen = np.zeros(a.n_states, dtype=bool)
        j = k
        while cur.size and j < n:
            nxt = a.delta[cur, w[j]]
            ok = nxt >= 0
            cur, start = nxt[ok], start[ok]
            hit = acc[cur]
            seen[start[hit]] = True
            j += 1
        out[k] = seen & qplus
    return out


def guarded_lex(dfa, data) -> Tuple[np.ndarray, np.ndarray, int, int]:
    """(kinds, lens, con, steps): the serial scan with each token ended as
    soon as the state leaves live_k."""
    a = _as_automaton(dfa)
    w = _as_bytes(data)
    n = int(w.size)
    live = live_sets(a, w)
    kinds, lens = [], []
    i, steps = 0, 0
    while i < n:
        q, j, last, kind = a.q0, i, None, -1
        while j < n and live[j, q]:
            t = int(a.delta[q, w[j]])
            steps += 1
            if t < 0:
                break
            q = t
            j += 1
            if a.tau[q] >= 0:
                last, kind = j, int(a.tau[q])
        if last is None:
            break
        kinds.append(kind)
        lens.append(last - i)
        i = last
    return np.asarray(kinds, np.int32), np.asarray(lens, np.int64), i, steps
