"""Pins of the liveness sets behind the failed-lookahead guard (no GPU).

live_k = { q in Q+ : delta*(q, w[k..m)) accepts for some m > k } (oracle/live.py).
Pinned against:
  * closed forms on the paper's example (Section 9: tokens a, a+b, ;) over
    a^n, a^n b and a^n ;, derived by hand from the three patterns;
  * Python's ``re`` for q0: q0 is live at k iff some token pattern fully
    matches some non-empty w[k..m), over every string up to length 6 on small
    alphabets of three token sets;
  * the maximal-munch scan: the scan that ends each token when its state
    leaves live_k gives exactly tok(w) and con(w) of the plain scan, in exactly
    con(w) transitions (a live state dropped from the sets would cut a token
    short; a dead one kept would cost steps);
  * the library's liveness automaton (lx_tokenset_liveness, host tables run
    from right to left in Python) gives the same sets.
"""

import itertools
import random
import re

import numpy as np
import pytest

import oracle
from oracle import live as L
from lexinputs import corpus
from lexinputs import tokensets as T


def _states(dfa):
    d = dfa.delta_full()
    q0 = dfa.q0
    A = int(d[q0, ord("a")])          # after one a: accepts a, continues a+b
    B = int(d[A, ord("a")])           # after two or more a: needs b
    C = int(d[A, ord("b")])           # a+b complete
    S = int(d[q0, ord(";")])
    return q0, A, B, C, S


def test_closed_forms_on_the_section9_example():
    dfa = T.tokenset("lookahead")
    q0, A, B, C, S = _states(dfa)
    assert int(dfa.delta_full()[B, ord("a")]) == B and int(dfa.delta_full()[B, ord("b")]) == C
    assert len({q0, A, B, C, S}) == 5
    n = 40
    # a^n: only q0 still meets an accepting state (the a token), never a b ahead
    lv = L.live_sets(dfa, b"a" * n)
    for k in range(n):
        assert set(np.flatnonzero(lv[k])) == {q0}, k
    assert not lv[n].any()
    # a^n b: q0, A and B all reach a+b (or a) before the end; at the b only A and B
    lv = L.live_sets(dfa, b"a" * n + b"b")
    for k in range(n):
        assert set(np.flatnonzero(lv[k])) == {q0, A, B}, k
    assert set(np.flatnonzero(lv[n])) == {A, B}
    assert not lv[n + 1].any()
    # a^n ; : the ; kills A and B, q0 accepts a (and ; at the last offset)
    lv = L.live_sets(dfa, b"a" * n + b";")
    for k in range(n + 1):
        assert set(np.flatnonzero(lv[k])) == {q0}, k


@pytest.mark.parametrize("name,alphabet", [("lookahead", b"ab;"), ("arith", b"a1=+ \n"), ("json", b'"a\\1.e-')])
def test_q0_liveness_matches_re(name, alphabet):
    tokens = T.token_list(name)
    pats = [re.compile(t.pattern.encode("latin-1")) for t in tokens]
    dfa = T.tokenset(name)
    for length in range(0, 7):
        strings = list(itertools.product(alphabet, repeat=length))
        if len(strings) > 4000:
            strings = random.Random(length).sample(strings, 4000)
        for tup in strings:
            w = bytes(tup)
            lv = L.live_sets(dfa, w)
            for k in range(len(w) + 1):
                want = any(p.fullmatch(w[k:m]) for m in range(k + 1, len(w) + 1) for p in pats)
                assert bool(lv[k, dfa.q0]) == want, (w, k)


@pytest.mark.parametrize("name", ["lookahead", "arith", "json", "clike", "clike_block"])
def test_guarded_scan_equals_the_serial_scan(name):
    rng = random.Random(77)
    dfa = T.tokenset(name)
    gen = {"lookahead": None, "clike_block": "clike_block"}.get(name, name)
    for trial in range(6):
        if gen is None:
            w = bytes(rng.choice(b"aaaab;") for _ in range(rng.randint(0, 300)))
        else:
            base = corpus.generate(gen, 3000, seed=trial)
            lo = rng.randrange(base.size)
            w = base[lo:lo + rng.randint(0, 600)].tobytes()
            if trial % 2 and w:
                pos = rng.randrange(len(w))
                w = w[:pos] + bytes([rng.choice(b"\x01?#")]) + w[pos + 1:]
        k1, l1, c1 = oracle.lex(dfa, w)
        k2, l2, c2, steps = L.guarded_lex(dfa, w)
        assert c1 == c2 and np.array_equal(k1, k2) and np.array_equal(l1, l2), (name, trial)
        assert steps == c1


def test_guard_makes_the_example_linear():
    dfa = T.tokenset("lookahead")
    for n in (50, 100, 200):
        k, l, con, steps = L.guarded_lex(dfa, b"a" * n)
        assert con == n and steps == n and (l == 1).all()


def _lib_sets(lg, name, w):
    """Sets of the library's liveness automaton, run from right to left."""
    ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    rc, blob, m = lg.lx_tokenset_liveness(ts)
    assert rc == 0
    R, C, S, W = m["R"], m["C"], m["S"], m["W"]
    cls = blob[:256]
    nxt = blob[m["next_off"]:m["next_off"] + C * R].reshape(C, R)
    mem = blob[m["member_off"]:m["member_off"] + 4 * R * W].view(np.uint32).reshape(R, W)
    out = np.zeros((len(w) + 1, S), dtype=bool)
    r = 0
    for k in range(len(w), -1, -1):
        if k < len(w):
            r = int(nxt[cls[w[k]], r])
        bits = mem[r]
        out[k] = [(int(bits[q >> 5]) >> (q & 31)) & 1 for q in range(S)]
    return out, blob, m


@pytest.mark.parametrize("name", ["lookahead", "arith", "json", "clike", "clike_block"])
def test_library_liveness_automaton_matches(lexlib, name):
    rng = random.Random(5)
    for trial in range(4):
        if name == "lookahead":
            w = bytes(rng.choice(b"aaab;") for _ in range(rng.randint(0, 200)))
        else:
            base = corpus.generate(name, 2000, seed=40 + trial)
            lo = rng.randrange(base.size)
            w = base[lo:lo + rng.randint(0, 300)].tobytes()
        got, blob, m = _lib_sets(lexlib, name, w)
        want = L.live_sets(T.tokenset(name), w)
        assert np.array_equal(got, want), (name, trial)


def test_library_reset_classes(lexlib):
    # a reset class maps every automaton state to the same state
    for name in ("json", "clike", "lookahead"):
        ts = lexlib.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
        rc, blob, m = lexlib.lx_tokenset_liveness(ts)
        R, C = m["R"], m["C"]
        nxt = blob[m["next_off"]:m["next_off"] + C * R].reshape(C, R)
        rst = blob[m["reset_off"]:m["reset_off"] + C]
        for c in range(C):
            assert bool(rst[c]) == (len(set(nxt[c].tolist())) == 1)
    # the newline resets the C-like automaton (no token spans a newline but ws)
    dfa = T.tokenset("clike")
    ts = lexlib.lx_compile_tokenset(dfa, T.discarded_kinds("clike"))
    rc, blob, m = lexlib.lx_tokenset_liveness(ts)
    assert blob[m["reset_off"] + int(dfa.byte_class[ord("\n")])] == 1
