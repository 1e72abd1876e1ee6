"""Independent pins of the oracle's pi_I (Section 5) and planner (Section 6).

Every expected stream and every expected cut list below is written out by
hand from the definitions, not computed by the oracle:

* pi_I deletes each (kind, length) pair whose kind lies in the discarded set
  I and keeps every other pair, in order, with its length unchanged (no
  merging of neighbours).
* the planner takes the k-1 equal-division targets t_i = floor(i n / k),
  slides each one forward to the next byte of the useful certified set (the
  chunk boundary lies just before that byte), drops targets that reach the
  end of the input or offset 0, and keeps each distinct offset once.
"""

import numpy as np

import oracle
from lexinputs import tokensets as T

# Figure 1: "int x=42;\nif(x)" under the arith token set
FIG1 = b"int x=42;\nif(x)"
FIG1_STREAM = [("ident", 3), ("space", 1), ("ident", 1), ("assign", 1), ("int", 2), ("semi", 1),
               ("newline", 1), ("ident", 2), ("lparen", 1), ("ident", 1), ("rparen", 1)]


def _ids(dfa, names):
    return [dfa.kind_names.index(x) for x in names]


def _stream(dfa, pairs):
    return (np.array([dfa.kind_names.index(k) for k, _ in pairs], np.int32),
            np.array([l for _, l in pairs], np.int64))


def _named(dfa, kinds, lens):
    return [(dfa.kind_names[int(k)], int(l)) for k, l in zip(kinds, lens)]


def test_discard_hand_streams_figure1():
    dfa = T.tokenset("arith")
    nk = len(dfa.kind_names)
    k, l = _stream(dfa, FIG1_STREAM)
    cases = {
        (): FIG1_STREAM,
        ("space",): [("ident", 3), ("ident", 1), ("assign", 1), ("int", 2), ("semi", 1), ("newline", 1),
                     ("ident", 2), ("lparen", 1), ("ident", 1), ("rparen", 1)],
        ("newline",): [("ident", 3), ("space", 1), ("ident", 1), ("assign", 1), ("int", 2), ("semi", 1),
                       ("ident", 2), ("lparen", 1), ("ident", 1), ("rparen", 1)],
        ("space", "newline"): [("ident", 3), ("ident", 1), ("assign", 1), ("int", 2), ("semi", 1),
                               ("ident", 2), ("lparen", 1), ("ident", 1), ("rparen", 1)],
        ("ident",): [("space", 1), ("assign", 1), ("int", 2), ("semi", 1), ("newline", 1), ("lparen", 1),
                     ("rparen", 1)],
        ("lparen", "rparen", "semi"): [("ident", 3), ("space", 1), ("ident", 1), ("assign", 1), ("int", 2),
                                       ("newline", 1), ("ident", 2), ("ident", 1)],
        tuple(dfa.kind_names): [],
    }
    for I, want in cases.items():
        ok, ol = oracle.discard(k, l, _ids(dfa, I), nk)
        assert _named(dfa, ok, ol) == want, I


def test_discard_of_the_serial_scan_figure1():
    # the composition pi_I(tok(w)) on the worked example, against the figure
    dfa = T.tokenset("arith")
    kinds, lens, con = oracle.lex(dfa, FIG1)
    assert con == len(FIG1)
    ok, ol = oracle.discard(kinds, lens, _ids(dfa, ["space", "newline"]), len(dfa.kind_names))
    assert _named(dfa, ok, ol) == [("ident", 3), ("ident", 1), ("assign", 1), ("int", 2), ("semi", 1),
                                   ("ident", 2), ("lparen", 1), ("ident", 1), ("rparen", 1)]


def test_discard_keeps_adjacent_discarded_runs_apart():
    # kinds 0 and 1 discarded; lengths of the kept pairs untouched, nothing merged
    k = np.array([0, 2, 1, 1, 3, 0, 2, 2, 1], np.int32)
    l = np.array([5, 1, 2, 3, 4, 6, 7, 8, 9], np.int64)
    ok, ol = oracle.discard(k, l, [0, 1], 4)
    assert ok.tolist() == [2, 3, 2, 2] and ol.tolist() == [1, 4, 7, 8]
    ok, ol = oracle.discard(k, l, [2], 4)
    assert ok.tolist() == [0, 1, 1, 3, 0, 1] and ol.tolist() == [5, 2, 3, 4, 6, 9]
    ok, ol = oracle.discard(k[:0], l[:0], [0], 4)
    assert ok.size == 0 and ol.size == 0


def _mask(*chars):
    m = np.zeros(256, bool)
    for c in chars:
        m[ord(c)] = True
    return m


def test_plan_hand_targets():
    semi = _mask(";")
    # n = 9, k = 3: targets 3, 6; 3 slides over 'c', 'd' to the ';' at 5, 6 is a ';'
    assert oracle.plan(b"ab;cd;;ef", semi, 3) == [5, 6]
    # targets 2, 4, 6 all slide to the one ';' at 8 (collisions kept once)
    assert oracle.plan(b"abcdefgh;", semi, 4) == [8]
    # certified byte at offset 0 is never a cut; n = 3, k = 8: targets 0,0,1,1,1,2,2
    assert oracle.plan(b";a;", semi, 8) == [2]
    # certified byte at offset n-1: the last chunk is that byte alone
    assert oracle.plan(b"abcdef;", semi, 2) == [6]
    # a target past the last certified byte slides off the end: no cut
    assert oracle.plan(b"a;bcdefg", semi, 2) == []
    # target 4 slides over "efg" to 7; a target that sits on a certified byte stays there
    assert oracle.plan(b"abc;efg;", semi, 2) == [7]
    assert oracle.plan(b"abcd;fgh", semi, 2) == [4]
    # k = 1, empty input, empty certified set: one chunk
    assert oracle.plan(b"a;b;c;d", semi, 1) == []
    assert oracle.plan(b"", semi, 4) == []
    assert oracle.plan(b"a;b;c;d", np.zeros(256, bool), 4) == []


def test_plan_several_certified_bytes():
    m = _mask("\n", "(", ")")
    w = b"x=1\nf(a)\n\nyy"          # n = 12
    # k = 4: targets 3, 6, 9 -> '\n' at 3, ')' at 7, '\n' at 9
    assert oracle.plan(w, m, 4) == [3, 7, 9]
    # k = 6: targets 2, 4, 6, 8, 10 -> 3, 5 ('('), 7, 8 ('\n'), 10 slides to 12 = n: dropped
    assert oracle.plan(w, m, 6) == [3, 5, 7, 8]
