"""Pins of the two-byte split windows (oracle/windows.py, no GPU).

cert(a, b): q0 not re-entrant, delta+(q0, b) defined, and no state of
Z(a) = delta+(Q+, a) has a live transition on b.  Pinned against:
  * Definition 2: b is exact-certified iff (a, b) is certified for every a
    (the union of Z(a) is every state inside a token), on every registered
    token set and on random automata;
  * the token boundary it promises: on every completely tokenizable string up
    to length 6 over small alphabets, every window cut is a boundary of tok(w);
  * Theorem 1's conclusion: scanning the chunks between window cuts and
    concatenating gives tok(w) and con(w), malformed strings included;
  * hand-worked JSON pairs;
  * the library's table (lx_window_certificates) equals the oracle's.
"""

import itertools
import random

import numpy as np
import pytest

import oracle
from oracle import windows as W
from lexinputs import corpus
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens

SETS = ["arith", "json", "clike", "clike_block", "lookahead", "utf8", "clike_row1"]


def _random_tokens(seed):
    rng = random.Random(seed)
    pats = []
    alpha = "abc;"
    for _ in range(rng.randint(2, 4)):
        body = "".join(rng.choice(alpha[:3]) for _ in range(rng.randint(1, 2)))
        pats.append(Token(f"t{len(pats)}", body + rng.choice(["", "+", "*"])))
    pats.append(Token("semi", ";"))
    pats.append(Token("sp", " +"))
    return pats


@pytest.mark.parametrize("name", SETS)
def test_definition_2_is_the_context_free_case(name):
    d = T.tokenset(name)
    cert = oracle.certificates(d)
    P = W.window_pairs(d)
    start = d.delta_full()[d.q0]
    for b in range(256):
        if start[b] < 0 or not cert.live[start[b]] or cert.reentrant:
            assert not P[:, b].any() or not cert.reentrant
            continue
        assert bool(cert.exact[b]) == bool(P[:, b].all()), (name, b)


@pytest.mark.parametrize("seed", range(12))
def test_definition_2_on_random_sets(seed):
    d = compile_tokens(_random_tokens(seed))
    cert = oracle.certificates(d)
    P = W.window_pairs(d)
    start = d.delta_full()[d.q0]
    for b in range(256):
        if cert.reentrant:
            assert not P.any()
            break
        if start[b] < 0 or not cert.live[start[b]]:
            assert not P[:, b].any()
            continue
        assert bool(cert.exact[b]) == bool(P[:, b].all())


@pytest.mark.parametrize("make", [T.ab_dead_chain, T.detached_state], ids=["ab_dead_chain", "detached_state"])
def test_definition_2_on_the_live_subautomaton_examples(make):
    # Section 4.1: states outside Q+ (a dead chain, a detached state) take no
    # part in Definition 2, nor in the window condition built on delta+
    d = make()
    cert = oracle.certificates(d)
    P = W.window_pairs(d)
    start = d.delta_full()[d.q0]
    assert not cert.reentrant and cert.exact.any()
    for b in range(256):
        if start[b] < 0 or not cert.live[start[b]]:
            assert not P[:, b].any()
            continue
        assert bool(cert.exact[b]) == bool(P[:, b].all()), b


def _boundaries(lens):
    return set(np.cumsum(lens).tolist()) | {0}


@pytest.mark.parametrize("name,alphabet", [("arith", b"a1=+ \n("), ("json", b'"a1 \n{}:,'),
                                           ("lookahead", b"ab; "), ("clike", b"a1 \n/\"=+")])
def test_window_cuts_are_token_boundaries(name, alphabet):
    d = T.tokenset(name)
    P = W.window_pairs(d)
    rng = random.Random(3)
    checked = 0
    for length in range(2, 7):
        strings = list(itertools.product(alphabet, repeat=length))
        if len(strings) > 6000:
            strings = rng.sample(strings, 6000)
        for tup in strings:
            w = bytes(tup)
            k, l, con = oracle.lex(d, w)
            if con != len(w):
                continue
            bounds = _boundaries(l)
            for p in W.window_cuts(d, w, P):
                assert p in bounds, (w, p)
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("seed", range(10))
def test_random_sets_boundaries_and_chunks(seed):
    d = compile_tokens(_random_tokens(100 + seed))
    P = W.window_pairs(d)
    for length in range(1, 7):
        for tup in itertools.product(b"abc; ", repeat=length):
            w = bytes(tup)
            cuts = W.window_cuts(d, w, P)
            k, l, con = oracle.lex(d, w)
            k2, l2, con2 = oracle.lex_chunks(d, w, cuts)
            assert con2 == con and np.array_equal(k, k2) and np.array_equal(l, l2), (w, cuts)


@pytest.mark.parametrize("name", ["json", "clike", "arith"])
def test_chunked_scan_at_window_cuts(name):
    d = T.tokenset(name)
    P = W.window_pairs(d)
    rng = random.Random(9)
    base = corpus.generate(name, 40_000, seed=5)
    for trial in range(12):
        lo = rng.randrange(base.size)
        w = base[lo:lo + rng.randint(1, 3000)].copy()
        if trial % 3 == 1 and w.size:
            w[rng.randrange(w.size)] = 0x01
        cuts = W.window_cuts(d, w, P)
        k, l, con = oracle.lex(d, w)
        k2, l2, con2 = oracle.lex_chunks(d, w, cuts)
        assert con2 == con and np.array_equal(k, k2) and np.array_equal(l, l2), (name, trial)


def test_json_pairs_by_hand():
    P = W.window_pairs(T.tokenset("json"))
    nl = ord("\n")
    # after a newline only a whitespace run can be in progress, and it cannot read a token's first byte
    for b in b'{}[]:,"-0123456789tfn':
        assert P[nl, b], chr(b)
    for b in b" \t\r\n":
        assert not P[nl, b]          # the whitespace run goes on
    assert not P[ord('"'), ord("{")]  # '"' may open a string that '{' continues
    assert not P[ord("a"), ord("b")]  # inside a string
    assert not P[ord("1"), ord("2")]  # inside a number
    # a ',' may sit inside a string, which the '"' then closes: the string token reads both
    assert not P[ord(","), ord('"')]
    # no JSON token holds a newline except a whitespace run, and none of these bytes starts or
    # continues one: the token before the newline ends there
    for a in b'}]"1e,:':
        assert P[a, nl], chr(a)


@pytest.mark.parametrize("name", SETS)
def test_library_table_matches(lexlib, name):
    ts = lexlib.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    rc, got = lexlib.lx_window_certificates(ts)
    assert rc == 0
    assert np.array_equal(got, W.window_pairs(T.tokenset(name)))
