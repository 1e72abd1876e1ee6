"""The CPU-parallel certified-split baseline (the paper's planner and executor
of Section 6 on host threads) gives the serial result: Theorem 1 for exact
cuts, Theorem 3 (pi_I) for modulo cuts, Corollary 1 on malformed input."""

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

CASES = [
    ("arith", "exact", False, 1 << 20),
    ("json", "modulo", True, 2 << 20),
    ("clike", "modulo", True, 2 << 20),
    ("clike_row1", "exact", False, 256 << 10),
]


def _serial(dfa, w, I):
    k, l, con = oracle.lex(dfa, w)
    if I:
        k, l = oracle.discard(k, l, I, len(dfa.kind_names))
    return k, l, con


@pytest.mark.parametrize("name,cert,filtered,n", CASES)
def test_par_lex_equals_serial(name, cert, filtered, n):
    dfa = T.tokenset(name)
    I = T.discarded_kinds(name) if filtered else []
    gen = "clike" if name == "clike_row1" else name
    w = corpus.generate(gen, n, seed=77).copy()
    c = oracle.certificates(dfa, I)
    useful = c.exact if cert == "exact" else c.modulo
    bad = w.copy()
    bad[n // 3] = 0x01                      # a lexing error one third in
    for data in (w, bad):
        rk, rl, rcon = _serial(dfa, data, I)
        for k in (1, 2, 3, 8, 17):
            ok, ol, con, chunks, sec = oracle.par_lex(dfa, data, useful, I, k)
            assert con == rcon
            assert np.array_equal(ok.astype(np.int64), rk.astype(np.int64))
            assert np.array_equal(ol.astype(np.int64), rl.astype(np.int64))
            assert 1 <= chunks <= k and sec >= 0.0


def test_par_lex_no_certified_byte_is_one_chunk():
    dfa = T.tokenset("json")
    w = corpus.generate("json", 64 << 10, seed=5)
    c = oracle.certificates(dfa, [])
    assert not c.exact.any()
    ok, ol, con, chunks, _ = oracle.par_lex(dfa, w, c.exact, [], 8)
    rk, rl, rcon = _serial(dfa, w, [])
    assert chunks == 1 and con == rcon and np.array_equal(ol.astype(np.int64), rl.astype(np.int64))


def test_par_lex_capacity_and_empty():
    dfa = T.tokenset("arith")
    c = oracle.certificates(dfa)
    w = corpus.generate("arith", 4096, seed=3)
    rk, rl, rcon = _serial(dfa, w, [])
    ok, ol, con, _, _ = oracle.par_lex(dfa, w, c.exact, [], 4, cap=rk.size)
    assert np.array_equal(ok.astype(np.int64), rk.astype(np.int64))
    with pytest.raises(ValueError):
        oracle.par_lex(dfa, w, c.exact, [], 4, cap=rk.size - 1)
    ok, ol, con, chunks, _ = oracle.par_lex(dfa, b"", c.exact, [], 4)
    assert ok.size == 0 and con == 0 and chunks == 1
