"""Two-byte split windows -- TEST INFRASTRUCTURE ONLY.

Sections 1 and 9 mention a generalisation of the certificate from single
bytes to short byte windows that certifies a cut at a fixed offset inside
every occurrence of a multi-byte string, the certificate of Definition 2
being its length-one case.  The paper gives no definition; this module holds
the one the library uses for windows of two bytes a b with the cut before b,
written out plainly:

    Z(a)      = { delta(q, a) : q in Q+, delta(q, a) in Q+ }
                (every state a scan can be in right after reading a, inside
                a token or having just started one: q0 is in Q+)
    cert(a,b) = q0 is not re-entrant  and  delta+(q0, b) is defined
                and  no state of Z(a) has a transition on b into Q+.

With q0 not re-entrant, no token can read a and then b: the token that
covers a ends at b's offset, so every occurrence of a b in a completely
tokenizable input puts a token boundary between them.  Without the context
(Z = Q+ minus q0, every state inside a token) the condition is Definition 2's
exact certificate restricted to useful bytes (Corollary 2); since the union
of Z(a) over all bytes a is exactly that set, b is exact-certified iff
(a, b) is certified for every a.

* ``window_pairs``  -- bool[256, 256]: cert(a, b) for every pair of bytes.
* ``window_cuts``   -- the offsets p (1 <= p < n) with cert(w[p-1], w[p]).
"""

from __future__ import annotations

from typing import List, Optional

import numpy as np

from . import _as_automaton, _as_bytes, certificates


def window_pairs(dfa) -> np.ndarray:
    a = _as_automaton(dfa)
    cert = certificates(a)
    live = np.asarray(cert.live, dtype=bool)
    out = np.zeros((256, 256), dtype=bool)
    if cert.reentrant or not live[a.q0]:
        return out

    def dplus(q: int, c: int) -> int:
        t = int(a.delta[q, c])
        return t if t >= 0 and live[q] and live[t] else -1

    states = [q for q in range(a.n_states) if live[q]]
    for x in range(256):
        Z = {dplus(q, x) for q in states} - {-1}
        for y in range(256):
            if dplus(a.q0, y) < 0:
                continue
            out[x, y] = all(dplus(z, y) < 0 for z in Z)
    return out


def window_cuts(dfa, data, pairs: Optional[np.ndarray] = None) -> List[int]:
    w = _as_bytes(data)
    P = window_pairs(dfa) if pairs is None else pairs
    return [p for p in range(1, int(w.size)) if P[w[p - 1], w[p]]]
