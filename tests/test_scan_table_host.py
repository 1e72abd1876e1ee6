"""Host-side check of the plain DFA scan table used by lx_lex_enumerative
(no GPU): candidate lists per byte against the oracle's candidates(b), the
next table against delta restricted to Q+, accept words against tau and the
discarded set."""

import numpy as np
import pytest

import oracle
from oracle import contexts as C
from lexinputs import tokensets as T

from test_oracle_bruteforce import _random_automata


def _u16(blob, off, n):
    return blob[off:off + 2 * n].view(np.uint16)


def _check(lg, dfa, discarded):
    ts = lg.lx_compile_tokenset(dfa, discarded)
    rc, blob, m = lg.lx_tokenset_scan_table(ts)
    assert rc == 0
    a = oracle.Automaton(dfa)
    S = a.n_states
    assert m["S"] == S and m["q0"] == a.q0
    live = C.live_states(a)
    cls = blob[:256]
    nxt = _u16(blob, m["next_off"], m["C"] * S).reshape(m["C"], S)
    for q in range(S):
        if not live[q]:
            continue
        for b in range(256):
            d = int(a.delta[q, b])
            want = (d | (0x8000 if a.tau[d] >= 0 else 0)) if (d >= 0 and live[d]) else 0xFFFF
            assert int(nxt[cls[b], q]) == want, (q, b)
    acc = _u16(blob, m["acc_off"], S)
    for q in range(S):
        k = int(a.tau[q])
        want = 0x7FFF if k < 0 else (k | (0 if k in discarded else 0x8000))
        assert int(acc[q]) == want
    cbeg = _u16(blob, m["cbeg_off"], 257)
    cand = _u16(blob, m["cand_off"], int(cbeg[256]))
    longest = 0
    for b in range(256):
        got = cand[cbeg[b]:cbeg[b + 1]].tolist()
        assert [C.BOUNDARY] + got == C.candidates(a, b, live), b
        longest = max(longest, len(got))
    assert m["max_cand"] == longest


@pytest.mark.parametrize("name", ["arith", "json", "clike", "clike_block", "utf8"])
def test_scan_table_token_sets(lexlib, name):
    _check(lexlib, T.tokenset(name), set(T.discarded_kinds(name)))


def test_scan_table_random_automata(lexlib):
    for i, dfa in enumerate(_random_automata(404, 20, 20)):
        disc = {0} if i % 3 == 0 and dfa.n_kinds > 1 else set()
        _check(lexlib, dfa, disc)
