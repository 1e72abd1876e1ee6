"""Host half of the C ABI (no GPU): lx_compile_tokenset's linear derivation
(Section 6 / 6.1) against the oracle's set-wise certificates."""

import random

import numpy as np
import pytest

import oracle
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens, dfa_from_edges


def _compare(lg, dfa, discarded):
    ts = lg.lx_compile_tokenset(dfa, discarded)
    ex, mo = lg.lx_certificates(ts)
    c = oracle.certificates(dfa, discarded)
    assert np.array_equal(ex, c.exact)
    assert np.array_equal(mo, c.modulo)
    info = lg.lx_tokenset_info(ts)
    assert info["n_live"] == int(c.live.sum())
    assert info["reentrant"] == c.reentrant
    return ts


@pytest.mark.parametrize("name", ["arith", "json", "clike", "clike_block", "clike_row1", "utf8"])
def test_registered_sets(lexlib, name):
    _compare(lexlib, T.tokenset(name), T.discarded_kinds(name))
    _compare(lexlib, T.tokenset(name), [])


def test_paper_examples(lexlib):
    _compare(lexlib, T.ab_dead_chain(), [])
    _compare(lexlib, T.detached_state(), [])
    for toks, I in [
        ([Token("a", "a+"), Token("s", ";")], []),
        ([Token("a", "a*")], [0]),
        ([Token("t", "(ab)*c")], []),
        ([Token("x", "ab*"), Token("y", "b+"), Token("c", "c")], [0, 1]),
        ([Token("ab", "ab")], []),
        ([Token("ba", "ba")], []),
    ]:
        _compare(lexlib, compile_tokens(toks), I)


def test_random_automata(lexlib):
    rng = random.Random(5)
    for _ in range(300):
        S = rng.randint(1, 8)
        alpha = b"abcd"
        edges = [(q, b, rng.randrange(S)) for q in range(S) for b in alpha if rng.random() < 0.5]
        acc = {q: rng.randrange(3) for q in range(S) if rng.random() < 0.4}
        dfa = dfa_from_edges(S, edges, acc, q0=rng.randrange(S), kind_names=["a", "b", "c"])
        I = [k for k in range(3) if rng.random() < 0.5]
        _compare(lexlib, dfa, I)


def test_validation_errors(lexlib):
    lg = lexlib
    good = T.tokenset("arith")

    class Bad:
        pass

    def make(**kw):
        b = Bad()
        b.n_states, b.q0, b.n_kinds = good.n_states, good.q0, good.n_kinds
        b.byte_class, b.next, b.accept = good.byte_class.copy(), good.next.copy(), good.accept.copy()
        for k, v in kw.items():
            setattr(b, k, v)
        return b

    with pytest.raises(lg.LexError) as e:
        lg.lx_compile_tokenset(make(q0=good.n_states))
    assert e.value.code == lg.LX_E_INVAL
    nxt = good.next.copy()
    nxt[0, 0] = good.n_states + 3
    with pytest.raises(lg.LexError):
        lg.lx_compile_tokenset(make(next=nxt))
    bc = good.byte_class.copy()
    bc[5] = good.n_classes
    with pytest.raises(lg.LexError):
        lg.lx_compile_tokenset(make(byte_class=bc))
    with pytest.raises(lg.LexError):
        lg.lx_compile_tokenset(good, [good.n_kinds])
    ts = lg.lx_compile_tokenset(good, [])
    assert ts.handle


def test_table_forms(lexlib):
    lg = lexlib
    for name, form in [("arith", 0), ("json", 0), ("clike", 1)]:
        ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
        for mode in range(3):
            info = lg.lx_tokenset_info(ts, mode)
            assert info["status"] == 0 and info["table_form"] == form, (name, mode, info)
