"""Framing at the producer (Section 7.1): a reserved byte with a rule of its
own certifies even for a token set whose certified sets are empty.

Pins (no GPU): the paper states that reserving 0x1E certifies a split symbol
for the block-comment row of Table 2 (whose certified sets are empty); the
library's framed token set and the oracle's certificates of an independently
built framed automaton both give exactly {0x1E}; by brute force on a tiny
token set, every occurrence of the reserved byte in a completely tokenizable
string begins a token, and the framed document with the frames deleted lexes
to the same kept tokens.
"""

import itertools

import numpy as np

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens

RS = T.FRAME


def _bytes(mask):
    return {b for b in range(256) if mask[b]}


def test_block_comment_row_gains_the_reserved_byte(lexlib):
    lg = lexlib
    dfa = T.tokenset("clike_block")
    plain = lg.lx_compile_tokenset(dfa, T.discarded_kinds("clike_block"))
    ex, mo = lg.lx_certificates(plain)
    assert not ex.any() and not mo.any()                 # Table 2: refused under both conditions
    framed = lg.lx_compile_tokenset_framed(dfa, T.discarded_kinds("clike_block"), RS, frame_discarded=True)
    ex, mo = lg.lx_certificates(framed)
    assert _bytes(ex) == {RS} and _bytes(mo) == {RS}
    c = oracle.certificates(T.framed(dfa), T.discarded_kinds("clike_block") + [dfa.n_kinds])
    assert _bytes(c.exact) == {RS} and _bytes(c.modulo) == {RS}


def test_framed_tiny_set_bruteforce():
    # tokens: a+, /*...*/ style comment over {a, *, /}, ';' -- then frame 'R'
    base = compile_tokens([Token("a", "a+", 0), Token("cmt", "/\\*([^*]|\\*+[^*/])*\\*+/", 0), Token("semi", ";", 0)])
    f = T.framed(base, ord("R"))
    c = oracle.certificates(f)
    assert _bytes(c.exact) == {ord("R")} | _bytes(oracle.certificates(base).exact)
    for L in range(1, 8):
        for t in itertools.product(b"a*/;R", repeat=L):
            w = bytes(t)
            k, l, con = oracle.lex(f, w)
            if con != L:
                continue
            starts = set(np.concatenate([[0], np.cumsum(l)[:-1]]).tolist())
            assert all(i in starts for i in range(L) if w[i] == ord("R")), w


def test_frames_sit_at_token_boundaries_of_the_unframed_stream():
    dfa = T.tokenset("clike_block")
    I = T.discarded_kinds("clike_block")
    w = corpus.generate("clike_block_framed", 1 << 20, seed=9)
    assert (w == RS).sum() > 1000
    f = T.framed(dfa)
    k, l, con = oracle.lex(f, w)
    assert con == w.size
    kf, lf = oracle.discard(k, l, I + [dfa.n_kinds], f.n_kinds)
    u = w[w != RS]
    ku, lu, conu = oracle.lex(dfa, u)
    ku, lu = oracle.discard(ku, lu, I, dfa.n_kinds)
    assert conu == u.size and np.array_equal(kf, ku) and np.array_equal(lf, lu)
