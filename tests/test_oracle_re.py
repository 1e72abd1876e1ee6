"""Cross-check of the oracle scanner (and of the automaton it is given)
against Python's ``re.fullmatch`` on short strings.

Longest match with the paper's tie rule (Section 3): at offset i take the
largest L such that some token's pattern matches w[i:i+L] exactly, and among
those the lowest (priority, token ID).  ``re`` evaluates the patterns
directly, with no automaton, so a wrong transition, a wrong tie-break, a lost
accepting position or a wrong restart offset in the oracle shows up here.
"""

import random
import re

import numpy as np
import pytest

import oracle
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens


def re_scan(tokens, w: bytes):
    pats = [re.compile(t.pattern.encode("latin-1")) for t in tokens]
    order = sorted(range(len(tokens)), key=lambda k: (tokens[k].priority, k))
    out = []
    i = 0
    while i < len(w):
        best = None
        for L in range(len(w) - i, 0, -1):
            for k in order:
                if pats[k].fullmatch(w[i:i + L]):
                    best = (k, L)
                    break
            if best:
                break
        if best is None:
            break
        out.append(best)
        i += best[1]
    return out, i


def _check(tokens, dfa, strings):
    for w in strings:
        ref, con = re_scan(tokens, w)
        k, l, c = oracle.lex(dfa, w)
        assert c == con, (w, c, con)
        assert list(zip(k.tolist(), l.tolist())) == ref, w


@pytest.mark.parametrize("name,alphabet", [
    ("arith", b"ab1 =+(;\n?"),
    ("json", b'{}[]:,"\\u0e1-.tn \n'),
    ("clike", b"ai0x.e+-<=>/\"'\\\n "),
    ("clike_block", b"a0/*\"\\\n "),
    ("utf8", bytes([0x41, 0xC3, 0xA9, 0xE0, 0xA0, 0x80, 0xF0, 0x90, 0xC0, 0xFF])),
])
def test_registered_sets_match_re(name, alphabet):
    rng = random.Random(1234)
    tokens = T.token_list(name)
    dfa = T.tokenset(name)
    strings = [bytes(rng.choice(alphabet) for _ in range(rng.randint(0, 9))) for _ in range(400)]
    _check(tokens, dfa, strings)


def _rand_regex(rng, depth=0):
    r = rng.random()
    if depth > 2 or r < 0.35:
        return rng.choice(["a", "b", "c", "[ab]", "[bc]", "[^a]"])
    if r < 0.55:
        return _rand_regex(rng, depth + 1) + _rand_regex(rng, depth + 1)
    if r < 0.7:
        return "(" + _rand_regex(rng, depth + 1) + "|" + _rand_regex(rng, depth + 1) + ")"
    q = rng.choice(["*", "+", "?"])
    return "(" + _rand_regex(rng, depth + 1) + ")" + q


def test_random_token_sets_match_re():
    rng = random.Random(99)
    for trial in range(60):
        n_tok = rng.randint(1, 4)
        toks = [Token(f"t{i}", _rand_regex(rng), rng.randint(0, 2)) for i in range(n_tok)]
        dfa = compile_tokens(toks)
        strings = [bytes(rng.choice(b"abcd") for _ in range(rng.randint(0, 7))) for _ in range(60)]
        _check(toks, dfa, strings)
