"""Pins of the entry-context oracle (splitting a refused token set).

Exhaustive on tiny automata (random regular-expression token sets and random
hand-assembled tables) and all strings over {a, b, c} up to length 6:

* the context at p is always among candidates(w[p-1]) (the enumeration is
  complete);
* chunk_run from the true context at p0 yields exactly the serial tokens that
  start in [p0, p1) and exits in the true context at p1 (or halts where the
  serial scan halts);
* chaining chunk runs reproduces tok(w), con(w) for every set of split points;
* where the serial scan is a plain longest-match over a single token (a* b
  style sets) contexts are the DFA states by hand;
* at an exactly certified byte of a tokenizable string the context is
  BOUNDARY (Lemma 1 in context form).
"""

import itertools
import random

import numpy as np

import oracle
from oracle import contexts as C
from lexinputs.automaton import Token, compile_tokens

from test_oracle_bruteforce import ALPHA, _random_automata, _strings


def _serial_starts(lens):
    return np.concatenate([[0], np.cumsum(lens)[:-1]]).tolist() if len(lens) else []


def test_context_always_a_candidate_and_chunk_runs_exact():
    for dfa in _random_automata(101, 25, 25):
        a = oracle.Automaton(dfa)
        live = C.live_states(a)
        cands = {b: set(C.candidates(a, b, live)) for b in ALPHA}
        for w in _strings(6):
            n = len(w)
            k, l, con = oracle.lex(a, w)
            ctx = C.contexts(a, w)
            starts = _serial_starts(l)
            for p in range(1, con + 1):
                assert ctx[p] in cands[w[p - 1]], (w, p, ctx[p])
            # every chunk [p0, p1) with p0 <= con, entered in the true context
            for p0 in range(0, con + 1):
                for p1 in range(p0 + 1, n + 1):
                    toks, ex, fail = C.chunk_run(a, w, p0, p1, ctx[p0])
                    assert toks is not None
                    want = [(int(kk), int(ll)) for kk, ll, s in zip(k, l, starts) if p0 <= s < p1]
                    assert toks == want, (w, p0, p1)
                    if con < n and p0 <= con < p1:
                        assert fail == con and ex is None, (w, p0, p1)
                    elif p1 <= con:
                        assert fail is None and ex == ctx[p1], (w, p0, p1, ex, ctx[p1])


def test_chained_runs_equal_serial_for_every_split_set():
    rng = random.Random(7)
    for dfa in _random_automata(202, 15, 15):
        a = oracle.Automaton(dfa)
        for w in _strings(5):
            k, l, con = oracle.lex(a, w)
            n = len(w)
            for r in range(0, n):
                for cuts in itertools.combinations(range(1, n), r):
                    if r > 2 and rng.random() < 0.7:
                        continue
                    k2, l2, c2 = C.chained(a, w, cuts)
                    assert c2 == con and np.array_equal(k2, k) and np.array_equal(l2, l), (w, cuts)


def test_contexts_by_hand():
    # one token a*b (kind 0) and single a (kind 1, priority lower): states
    # q0 -a-> qa (accepting kind 1) -a-> qaa -b-> qb; longest match
    dfa = compile_tokens([Token("ab", "a*b", 0), Token("a", "a", 1)])
    a = oracle.Automaton(dfa)
    w = b"aaab"
    ctx = C.contexts(a, w)
    assert ctx[0] == C.BOUNDARY and ctx[4] == C.BOUNDARY
    q = a.q0
    for p in range(1, 4):
        q = int(a.delta[q, w[p - 1]])
        assert ctx[p] == q                    # inside the single token [0, 4)
    # "aac": a*b never completes, so the scan backtracks to "a" twice and
    # halts before 'c' (in neither token's alphabet)
    k, l, con = oracle.lex(a, b"aac")
    assert con == 2 and l.tolist() == [1, 1]
    assert C.contexts(a, b"aac")[:3] == [C.BOUNDARY, C.BOUNDARY, C.BOUNDARY]
    # a wrong mid-token guess that can never accept is reported as invalid
    dead_guess = int(a.delta[a.q0, ord("a")])
    toks, ex, fail = C.chunk_run(a, b"aac", 2, 3, dead_guess)
    assert toks is None


def test_certified_bytes_have_boundary_context():
    for dfa in _random_automata(303, 30, 30):
        a = oracle.Automaton(dfa)
        cert = oracle.certificates(a)
        exact = {b for b in ALPHA if cert.exact[b]}
        if not exact:
            continue
        for w in _strings(6):
            k, l, con = oracle.lex(a, w)
            if con != len(w):
                continue
            ctx = C.contexts(a, w)
            for p, b in enumerate(w):
                if b in exact:
                    assert ctx[p] == C.BOUNDARY, (w, p)
