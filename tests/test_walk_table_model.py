"""Host-side check of the packed walk tables (no GPU).

The device kernel plans one chunk start per SEG-byte target (the first
certified byte of the segment), walks each range over the Moore-form table
of ``lx_tokenset_table`` and concatenates the ranges in order.  This test
replays exactly that table semantics in Python on small inputs, with tiny
segments so that every cut and range boundary is exercised, and compares the
result with the oracle (tok(w) in full or pi_I(tok(w)), and con(w)).  A
wrong row target, kind word, cut flag or pointer encoding in the table
builder shows up here before any GPU run.
"""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

NOPOS = None


class TableModel:
    def __init__(self, lg, ts, mode, class_table=False):
        rc, blob, info = lg.lx_tokenset_table(ts, mode, class_table)
        assert rc == 0
        self.b = blob
        self.i = info
        self.u16 = lambda off: int(self.b[off]) | (int(self.b[off + 1]) << 8)
        self.cert = blob[info["cert_off"]:info["cert_off"] + 256].astype(bool)
        self.cmap = blob[info["cmap_off"]:info["cmap_off"] + 256]

    def step(self, e, b):
        if self.i["form"] == 0:
            return self.u16(e ^ (b << 1))
        return self.u16(e + 2 * int(self.cmap[b]))

    def kind(self, e):
        if self.i["form"] == 0:
            return self.u16(self.i["kind_off"] + 2 * (e >> 9))
        return self.u16(e + 2 * (self.i["ncols"] - 1))

    def walk(self, w, start, seg_end, out):
        """Mirror of the kernel's walk(); returns the failure offset or None."""
        n = len(w)
        P_start, P_flag, P_slow = self.i["p_start"], self.i["p_flag"], self.i["p_slow"]
        p = tok = start
        e = P_start
        while True:
            slow = False
            if p == n:
                if e == P_start:
                    return None
                kw = self.kind(e)
                if (kw & 0x7FFF) != 0x7FFF:
                    self.emit(out, kw, p - tok)
                    return None
                slow = True
            else:
                b = w[p]
                e2 = self.step(e, b)
                if e2 == P_slow:
                    slow = True
                elif e2 >= P_flag:
                    if True:
                        self.emit(out, self.kind(e), p - tok)
                        tok = p
                        if p >= seg_end and self.cert[b]:
                            return None
                if not slow:
                    e = e2
                    p += 1
                    continue
            q, r, rk = P_start, None, 0
            for j in range(tok, p):
                q = self.step(q, w[j])
                kw = self.kind(q)
                if (kw & 0x7FFF) != 0x7FFF:
                    r, rk = j + 1, kw
            if r is None:
                return tok
            self.emit(out, rk, r - tok)
            tok = p = r
            e = P_start
            if r == n:
                return None
            if r >= seg_end and self.cert[w[r]]:
                return None

    @staticmethod
    def emit(out, kw, length):
        if kw & 0x8000:
            out.append((kw & 0x7FFF, length))

    def lex(self, w, seg):
        n = len(w)
        tokens, fail = [], None
        for t in range(0, max(1, -(-n // seg))):
            s0 = t * seg
            start = 0 if t == 0 else next((p for p in range(s0, min(s0 + seg, n)) if self.cert[w[p]]), None)
            if start is None:
                continue
            out = []
            f = self.walk(w, start, s0 + seg, out)
            tokens += out
            if f is not None:
                return tokens, f
        return tokens, n


def _expected(dfa, w, mode, discarded):
    k, l, con = oracle.lex(dfa, w)
    if mode != 0:
        k, l = oracle.discard(k, l, discarded, dfa.n_kinds)
    return list(zip(k.tolist(), l.tolist())), con


@pytest.mark.parametrize("class_table", [False, True])
@pytest.mark.parametrize("name", ["arith", "json", "clike", "clike_row1"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_table_model_matches_oracle(lexlib, name, mode, class_table):
    if mode == 0 and name in ("json", "clike"):
        seg_list = [7]
    else:
        seg_list = [1, 3, 7, 68]
    dfa = T.tokenset(name)
    I = T.discarded_kinds(name)
    ts = lexlib.lx_compile_tokenset(dfa, I)
    m = TableModel(lexlib, ts, mode, class_table)
    if class_table:
        assert m.i["form"] == 1
    rng = random.Random(hash((name, mode)) & 0xFFFF)
    wl = {"arith": "arith", "json": "json", "clike": "clike", "clike_row1": "clike"}[name]
    base = bytes(corpus.generate(wl, 1 << 15, seed=11))
    cases = [base[:0], base[:1], base[:2000]]
    for _ in range(25):
        a = rng.randrange(0, len(base) - 400)
        s = bytearray(base[a:a + rng.randint(1, 400)])
        if rng.random() < 0.3 and s:                      # inject a malformed byte
            s[rng.randrange(len(s))] = rng.choice(b"\x01`@#$\x7f")
        cases.append(bytes(s))
    for w in cases:
        exp = _expected(dfa, w, mode, I)
        for seg in seg_list:
            got = m.lex(w, seg)
            assert got[1] == exp[1], (name, mode, seg, w[:80])
            assert got[0] == exp[0], (name, mode, seg, w[:80])


def wide_class_dfa(seed=5, n_states=12, n_bytes=150):
    """A DFA whose bytes fall into more than 128 classes (each byte maps the
    states differently) with few states."""
    from lexinputs.automaton import dfa_from_edges
    rng = random.Random(seed)
    alpha = list(range(32, 32 + n_bytes))
    edges = []
    for q in range(n_states):
        for b in alpha:
            if q == 0 or rng.random() < 0.7:
                edges.append((q, b, rng.randrange(1, n_states)))
    acc = {q: rng.randrange(3) for q in range(1, n_states)}
    return dfa_from_edges(n_states, edges, acc, q0=0, kind_names=["k0", "k1", "k2"]), alpha


def test_wide_class_table_model(lexlib):
    dfa, alpha = wide_class_dfa()
    assert dfa.n_classes > 128
    ts = lexlib.lx_compile_tokenset(dfa, [1])
    rng = random.Random(6)
    for mode in (0, 1):
        m = TableModel(lexlib, ts, mode, class_table=True)
        assert m.i["form"] == 1
        for _ in range(30):
            w = bytes(rng.choice(alpha) for _ in range(rng.randint(0, 300)))
            exp = _expected(dfa, w, mode, [1])
            for seg in (3, 7, 68):
                got = m.lex(w, seg)
                assert got[1] == exp[1] and got[0] == exp[0]
