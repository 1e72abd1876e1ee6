"""Pins of the CPU oracle against values the paper prints or fixes.

Each test names the passage it follows.  These run without a GPU.
"""

import os

import numpy as np
import pytest

import oracle
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _set(*chars):
    out = set()
    for c in chars:
        out.add(c if isinstance(c, int) else ord(c))
    return out


def _bytes_of(mask):
    return {b for b in range(256) if mask[b]}


def _compile(*specs):
    return compile_tokens([Token(n, p, pr) for (n, p, pr) in specs])


# --- Figure 1: the worked split ------------------------------------------------

def test_figure1_extents_and_split():
    fields = {}
    with open(os.path.join(GOLDEN, "fig1_split.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(" ", 1)
            fields[k] = v.strip()
    w = bytes.fromhex(fields["input_hex"])
    extents = [tuple(int(x) for x in e.split("-")) for e in fields["extents"].split()]
    cut = int(fields["certified_offset"])
    dfa = T.tokenset("arith")
    kinds, lens, con = oracle.lex(dfa, w)
    assert con == len(w)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    assert [(int(s), int(s + l - 1)) for s, l in zip(starts, lens)] == extents
    assert [dfa.kind_names[k] for k in kinds] == [
        "ident", "space", "ident", "assign", "int", "semi", "newline", "ident", "lparen",
        "ident", "rparen"]
    cert = oracle.certificates(dfa)
    assert cert.exact[w[cut]]
    k2, l2, con2 = oracle.lex_chunks(dfa, w, [cut])
    assert con2 == len(w) and list(k2) == list(kinds) and list(l2) == list(lens)


# --- Figure 2 and Section 4.2: the re-entrancy subtlety -------------------------

def test_figure2a_aplus_semicolon():
    dfa = _compile(("a", "a+", 0), ("semi", ";", 0))
    c = oracle.certificates(dfa)
    assert not c.reentrant
    assert _bytes_of(c.exact) == _set(";")


def test_nullable_astar_is_reentrant_and_refused():
    dfa = _compile(("a", "a*", 0))
    assert dfa.n_states == 1 and dfa.accept[0] == 0          # one accepting self-looping state
    c = oracle.certificates(dfa)
    assert c.reentrant
    assert not c.exact[ord("a")]
    # the naive criterion (only q0 consumes 'a') would admit it, and splitting "aa"
    # there gives two tokens where the serial scan gives one
    assert oracle.lex(dfa, b"aa")[0].size == 1
    assert oracle.lex_chunks(dfa, b"aa", [1])[0].size == 2


def test_cyclic_abstar_c_reentrant_without_self_loop():
    dfa = _compile(("t", "(ab)*c", 0))
    delta = dfa.delta_full()
    assert all(delta[q, b] != q for q in range(dfa.n_states) for b in range(256))
    c = oracle.certificates(dfa)
    assert c.reentrant
    assert not c.exact[ord("c")]
    # only q0 consumes 'c'
    consumers = {q for q in range(dfa.n_states) if delta[q, ord("c")] >= 0}
    assert consumers == {dfa.q0}
    k, l, con = oracle.lex(dfa, b"abc")
    assert con == 3 and list(l) == [3]


# --- Section 4.1: restricting to the live subautomaton ---------------------------

def test_dead_chain_ab_emptyset_beside_b():
    dfa = T.ab_dead_chain()
    c = oracle.certificates(dfa)
    assert list(np.nonzero(c.live)[0]) == [0, 3]
    assert c.exact[ord("b")]                     # certified and useful
    assert c.exact_raw[ord("a")] and not c.exact[ord("a")]   # vacuous, withheld


def test_detached_state_does_not_decertify():
    dfa = T.detached_state()
    c = oracle.certificates(dfa)
    assert not c.live[4] and not c.live[5]
    assert c.exact[ord("b")]


# --- Section 4: UTF-8 encoding forms ---------------------------------------------

def test_utf8_forms_byte_for_byte():
    c = oracle.certificates(T.tokenset("utf8"))
    expect = set(range(0x00, 0x80)) | set(range(0xC2, 0xE0)) | set(range(0xE0, 0xF0)) | \
        set(range(0xF0, 0xF5))
    assert _bytes_of(c.exact) == expect
    assert not any(c.exact[b] for b in range(0x80, 0xC0))
    vacuous = {0xC0, 0xC1} | set(range(0xF5, 0x100))
    assert all(c.exact_raw[b] and not c.exact[b] for b in vacuous)


# --- Section 5: certification modulo discarded tokens -----------------------------

def test_discarded_astar_certified_modulo():
    dfa = _compile(("a", "a*", 0))
    c = oracle.certificates(dfa, [0])
    assert c.reentrant
    assert _bytes_of(c.modulo) == _set("a")
    assert _bytes_of(c.exact) == set()


def test_prop3_strict_extension_newline():
    dfa = _compile(("ident", "[a-z]+", 0), ("semi", ";", 0), ("lp", "\\(", 0),
                   ("ws", "[ \\n]+", 0))
    ws = dfa.kind_id("ws")
    c = oracle.certificates(dfa, [ws])
    assert not c.exact[ord("\n")]
    assert c.modulo[ord("\n")]
    assert _bytes_of(c.exact) <= _bytes_of(c.modulo)


def test_line_comment_is_not_enough():
    # cutting //ab between its last two bytes leaves a comment and an identifier
    dfa = _compile(("ident", "[a-z]+", 0), ("slash", "/", 0), ("comment", "//[a-z]*", 0))
    c = oracle.certificates(dfa, [dfa.kind_id("comment")])
    assert not c.modulo[ord("b")]


def test_conservativeness_witness():
    dfa = _compile(("abstar", "ab*", 0), ("bplus", "b+", 0), ("c", "c", 0))
    I = [0, 1]
    c = oracle.certificates(dfa, I)
    assert not c.modulo[ord("b")]        # condition 2 fails
    # ... yet every occurrence of b is safe modulo I (bounded form, length <= 6)
    import itertools
    for L in range(1, 7):
        for t in itertools.product(b"abc", repeat=L):
            w = bytes(t)
            k, l, con = oracle.lex(dfa, w)
            if con != L:
                continue
            cuts = [i for i in range(1, L) if w[i] == ord("b")]
            k2, l2, con2 = oracle.lex_chunks(dfa, w, cuts)
            assert con2 == L
            a = oracle.discard(k, l, I, 3)
            b = oracle.discard(k2, l2, I, 3)
            assert list(a[0]) == list(b[0]) and list(a[1]) == list(b[1])


def _every_cut_keeps_pi_I(dfa, I, alphabet, byte, max_len):
    """Bounded soundness: on every string over `alphabet` up to `max_len` bytes,
    the chunked scan cut before every occurrence of `byte` gives pi_I of the
    serial scan and the same consumed length (Theorem 3 and Corollary 1)."""
    import itertools
    nk = dfa.n_kinds
    for L in range(1, max_len + 1):
        for t in itertools.product(alphabet, repeat=L):
            w = bytes(t)
            k, l, con = oracle.lex(dfa, w)
            cuts = [i for i in range(1, con) if w[i] == byte]
            k2, l2, con2 = oracle.lex_chunks(dfa, w[:con], cuts)
            a, b = oracle.discard(k, l, I, nk), oracle.discard(k2, l2, I, nk)
            if con2 != con or list(a[0]) != list(b[0]) or list(a[1]) != list(b[1]):
                return w
    return None


def test_modulo_needs_an_accepting_state():
    # Definition 3, C(q) asks for tau(q) defined: in the discarded token a?b+
    # the state after 'a' is not accepting, goes to the same state on 'b' as
    # q0 and reaches only discarded kinds, yet a cut before the 'b' of "ab"
    # leaves the chunk "a", which does not lex
    dfa = _compile(("d", "a?b+", 0), ("semi", ";", 0))
    I = [dfa.kind_id("d")]
    c = oracle.certificates(dfa, I)
    assert not c.modulo[ord("b")]
    assert oracle.lex(dfa, b"ab")[2] == 2 and oracle.lex_chunks(dfa, b"ab", [1])[2] == 0
    assert _every_cut_keeps_pi_I(dfa, I, b"ab;", ord("b"), 6) == b"ab"


def test_modulo_through_a_non_accepting_inner_state():
    # Definition 3, T(q) collects the kinds of the ACCEPTING states reachable
    # from q: whitespace with line continuations (runs of spaces and of a
    # backslash followed by a newline) passes through the non-accepting state
    # after the backslash, and ' ' is still certified modulo I = {ws} --
    # soundly, by the bounded check
    dfa = _compile(("x", "x+", 0), ("ws", "( |\\\\\n)+", 0))
    delta = dfa.delta_full()
    after_bs = [q for q in range(dfa.n_states) if q != dfa.q0 and delta[q, ord("\\")] >= 0]
    assert after_bs and all(dfa.accept[delta[q, ord("\\")]] < 0 for q in after_bs)
    I = [dfa.kind_id("ws")]
    c = oracle.certificates(dfa, I)
    assert not c.exact[ord(" ")]
    assert c.modulo[ord(" ")]
    assert _every_cut_keeps_pi_I(dfa, I, b"x \\\n", ord(" "), 6) is None


def test_empty_discard_set_recovers_exact():
    # Section 5: with I empty no accepting state has T(q) inside I, so C(q)
    # never holds and Definition 3 reduces to Definition 2 -- also when q0 is
    # re-entrant, where A(q0) fails and the byte stays refused
    sets = [(name, T.tokenset(name)) for name in ("arith", "json", "clike", "clike_row1", "utf8")]
    sets += [("a*", _compile(("a", "a*", 0))), ("(ab)*c", _compile(("t", "(ab)*c", 0)))]
    for name, dfa in sets:
        c = oracle.certificates(dfa, [])
        assert np.array_equal(c.exact_raw, c.modulo_raw), name
        assert np.array_equal(c.exact, c.modulo), name
    assert not oracle.certificates(sets[-2][1], []).modulo_raw[ord("a")]
    assert not oracle.certificates(sets[-1][1], []).modulo_raw[ord("c")]


# --- Section 8: re2c sentinel contrast ---------------------------------------------

def test_re2c_contrast():
    c_ab = oracle.certificates(_compile(("ab", "ab", 0)))
    c_ba = oracle.certificates(_compile(("ba", "ba", 0)))
    assert not c_ab.exact[ord("b")]
    assert c_ba.exact[ord("b")]


# --- Section 7: quadratic failed lookahead ---------------------------------------------

def test_quadratic_lookahead_set():
    dfa = _compile(("a", "a", 0), ("apb", "a+b", 0), ("semi", ";", 0))
    c = oracle.certificates(dfa)
    assert _bytes_of(c.exact) == _set(";")
    w = b"a" * 300
    k, l, con = oracle.lex(dfa, w)
    assert con == 300 and k.size == 300 and set(l.tolist()) == {1}
    assert oracle.plan(w, c.exact, 8) == []      # never occurs: one chunk


# --- Table 2 rows ------------------------------------------------------------------

@pytest.mark.parametrize("name,exact,modulo", [
    ("json", set(), _set("\t", "\n", "\r")),
    ("clike", set(), _set("\n")),
    ("clike_block", set(), set()),
    ("clike_row1", set(map(ord, "+-*/%=<>!&|^~?:;,.()[]{}")),
     set(map(ord, "+-*/%=<>!&|^~?:;,.()[]{}")) | _set(" ", "\t", "\n")),
])
def test_table2_rows(name, exact, modulo):
    c = oracle.certificates(T.tokenset(name), T.discarded_kinds(name))
    assert _bytes_of(c.exact) == exact
    assert _bytes_of(c.modulo) == modulo


def test_arith_set_certificates():
    # By Definition 2 the single-byte operators consumed only at q0 certify;
    # '=' is continued by '==' and a space by its run.
    c = oracle.certificates(T.tokenset("arith"))
    assert _bytes_of(c.exact) == set(map(ord, "\n()*+-/;"))
    assert not c.exact[ord("=")] and not c.exact[ord(" ")]


# --- Corollary 1: malformed input ---------------------------------------------------

def test_malformed_input_prefix():
    dfa = T.tokenset("arith")
    w = b"ab+cd;\nx=1?y;\nz(2)\n"
    k, l, con = oracle.lex(dfa, w)
    assert con == w.index(b"?")
    c = oracle.certificates(dfa)
    cuts = [i for i in range(1, len(w)) if c.exact[w[i]]]
    k2, l2, con2 = oracle.lex_chunks(dfa, w, cuts)
    assert con2 == con and list(k2) == list(k) and list(l2) == list(l)


def test_scanner_edge_cases():
    dfa = T.tokenset("arith")
    assert oracle.lex(dfa, b"")[2] == 0
    k, l, con = oracle.lex(dfa, b"?")
    assert con == 0 and k.size == 0
    # longest match with backtracking: '=' then '=' + ... ; '==' wins when present
    k, l, con = oracle.lex(dfa, b"===")
    assert [dfa.kind_names[x] for x in k] == ["eq", "assign"] and list(l) == [2, 1]


def test_backtracking_clike_ellipsis():
    dfa = T.tokenset("clike")
    k, l, con = oracle.lex(dfa, b"a..b")
    names = [dfa.kind_names[x] for x in k]
    assert names == ["ident", "op6_.", "op6_.", "ident"] and con == 4
    k, l, con = oracle.lex(dfa, b"0x")
    assert [dfa.kind_names[x] for x in k] == ["int", "ident"]
