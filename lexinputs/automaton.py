"""Token-set specifications compiled to deterministic partial automata.

This module is part of the seeded input generators.  It turns a list of token
patterns into the compiled automaton A = (Q, Sigma, delta, q0, tau) that the
paper takes as given (Section 3): a partial transition function over the byte
alphabet, an initial state, and a partial accepting map whose value already
holds the winner of any same-length tie (lower priority number first, lower
token ID second).  It performs no certificate analysis and no scanning; both
the CPU oracle and the GPU library receive its output as *input*.

Pipeline: regular expression -> Thompson NFA -> subset construction over
byte classes -> partition-refinement minimisation that keeps a missing
transition distinct from a transition into a state that cannot accept (the
minimiser semantics of Section 4.1; deliberately weaker than Myhill-Nerode,
so chains of dead states survive) -> byte-class merging.

Supported pattern syntax (a subset that Python's ``re`` reads the same way
over bytes): literals, escapes ``\\n \\t \\r \\v \\f \\xHH`` and escaped
punctuation, classes ``[...]`` / ``[^...]`` with ranges, grouping ``( )``,
alternation ``|`` and the quantifiers ``* + ? {m} {m,} {m,n}``.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ALL_BYTES = (1 << 256) - 1
UNDEF = -1

_ESCAPES = {"n": 10, "t": 9, "r": 13, "v": 11, "f": 12, "0": 0, "a": 7, "e": 27}


def _byte_mask(lo: int, hi: int) -> int:
    return ((1 << (hi + 1)) - 1) ^ ((1 << lo) - 1)


class _Parser:
    """Recursive-descent parser producing a small syntax tree."""

    def __init__(self, pattern: str):
        self.s = pattern
        self.i = 0

    def error(self, msg: str) -> ValueError:
        return ValueError(f"pattern {self.s!r} at {self.i}: {msg}")

    def peek(self) -> Optional[str]:
        return self.s[self.i] if self.i < len(self.s) else None

    def take(self) -> str:
        if self.i >= len(self.s):
            raise self.error("unexpected end")
        c = self.s[self.i]
        self.i += 1
        return c

    def parse(self):
        node = self.alternation()
        if self.i != len(self.s):
            raise self.error("trailing input")
        return node

    def alternation(self):
        branches = [self.sequence()]
        while self.peek() == "|":
            self.i += 1
            branches.append(self.sequence())
        return branches[0] if len(branches) == 1 else ("alt", branches)

    def sequence(self):
        items = []
        while self.peek() is not None and self.peek() not in "|)":
            items.append(self.repetition())
        return ("seq", items)

    def repetition(self):
        node = self.atom()
        while self.peek() is not None and self.peek() in "*+?{":
            c = self.take()
            if c == "*":
                node = ("rep", node, 0, None)
            elif c == "+":
                node = ("rep", node, 1, None)
            elif c == "?":
                node = ("rep", node, 0, 1)
            else:
                j = self.s.index("}", self.i)
                body = self.s[self.i:j]
                self.i = j + 1
                if "," in body:
                    lo_s, hi_s = body.split(",", 1)
                    lo = int(lo_s)
                    hi = int(hi_s) if hi_s.strip() else None
                else:
                    lo = hi = int(body)
                node = ("rep", node, lo, hi)
        return node

    def escape_value(self) -> int:
        c = self.take()
        if c == "x":
            h = self.s[self.i:self.i + 2]
            self.i += 2
            return int(h, 16)
        if c in _ESCAPES:
            return _ESCAPES[c]
        if c.isalnum():
            raise self.error(f"unsupported escape \\{c}")
        return ord(c)

    def char_value(self) -> int:
        c = self.take()
        if c == "\\":
            return self.escape_value()
        v = ord(c)
        if v > 255:
            raise self.error("non-byte character")
        return v

    def atom(self):
        c = self.peek()
        if c == "(":
            self.i += 1
            node = self.alternation()
            if self.take() != ")":
                raise self.error("expected )")
            return node
        if c == "[":
            self.i += 1
            negate = False
            if self.peek() == "^":
                negate = True
                self.i += 1
            mask = 0
            first = True
            while True:
                if self.peek() == "]" and not first:
                    self.i += 1
                    break
                first = False
                lo = self.char_value()
                if self.peek() == "-" and self.s[self.i + 1:self.i + 2] not in ("]", ""):
                    self.i += 1
                    hi = self.char_value()
                    if hi < lo:
                        raise self.error("bad range")
                    mask |= _byte_mask(lo, hi)
                else:
                    mask |= 1 << lo
            if negate:
                mask = ALL_BYTES & ~mask
            return ("set", mask)
        if c == "\\":
            self.i += 1
            return ("set", 1 << self.escape_value())
        if c in ")*+?{}|]^$.":
            raise self.error(f"unexpected {c!r}")
        self.i += 1
        v = ord(c)
        if v > 255:
            raise self.error("non-byte character")
        return ("set", 1 << v)


class _NFA:
    def __init__(self):
        self.eps: List[List[int]] = []
        self.edges: List[List[Tuple[int, int]]] = []

    def new(self) -> int:
        self.eps.append([])
        self.edges.append([])
        return len(self.eps) - 1

    def build(self, node) -> Tuple[int, int]:
        kind = node[0]
        if kind == "set":
            a, b = self.new(), self.new()
            self.edges[a].append((node[1], b))
            return a, b
        if kind == "seq":
            a = self.new()
            cur = a
            for item in node[1]:
                s, e = self.build(item)
                self.eps[cur].append(s)
                cur = e
            return a, cur
        if kind == "alt":
            a, b = self.new(), self.new()
            for br in node[1]:
                s, e = self.build(br)
                self.eps[a].append(s)
                self.eps[e].append(b)
            return a, b
        if kind == "rep":
            _, sub, lo, hi = node
            a = self.new()
            cur = a
            for _ in range(lo):
                s, e = self.build(sub)
                self.eps[cur].append(s)
                cur = e
            if hi is None:
                s, e = self.build(sub)
                loop_in = self.new()
                self.eps[cur].append(loop_in)
                self.eps[loop_in].append(s)
                self.eps[e].append(loop_in)
                out = self.new()
                self.eps[loop_in].append(out)
                return a, out
            out = self.new()
            self.eps[cur].append(out)
            for _ in range(hi - lo):
                s, e = self.build(sub)
                self.eps[cur].append(s)
                self.eps[e].append(out)
                cur = e
            return a, out
        raise ValueError(kind)


@dataclass(frozen=True)
class Token:
    """One token kind.  ``kind`` is its token ID (order of definition)."""
    name: str
    pattern: str
    priority: int = 0


@dataclass
class DFA:
    """A deterministic partial automaton over bytes.

    ``next[c][q]`` is the target of state ``q`` on any byte of class ``c``
    (``UNDEF`` when the transition is missing); ``accept[q]`` is the token
    kind accepted in ``q`` or ``UNDEF``.
    """
    n_states: int
    q0: int
    byte_class: np.ndarray          # uint8[256] (class ids < 256)
    next: np.ndarray                # int32[n_classes, n_states]
    accept: np.ndarray              # int32[n_states]
    kind_names: List[str] = field(default_factory=list)

    @property
    def n_classes(self) -> int:
        return int(self.next.shape[0])

    @property
    def n_kinds(self) -> int:
        if self.kind_names:
            return len(self.kind_names)
        return int(self.accept.max()) + 1 if (self.accept >= 0).any() else 0

    def delta_full(self) -> np.ndarray:
        """int32[n_states, 256]: delta(q, b), UNDEF where undefined."""
        return np.ascontiguousarray(self.next[self.byte_class.astype(np.int64), :].T.astype(np.int32))

    def kind_id(self, name: str) -> int:
        return self.kind_names.index(name)


def dfa_from_full_table(delta: Sequence[Sequence[int]], accept: Sequence[int], q0: int = 0,
                        kind_names: Optional[List[str]] = None) -> DFA:
    """Wrap a hand-written ``delta[q][b]`` table (no minimisation)."""
    d = np.asarray(delta, dtype=np.int32)
    assert d.ndim == 2 and d.shape[1] == 256
    cols: Dict[bytes, int] = {}
    byte_class = np.zeros(256, dtype=np.uint8)
    uniq = []
    for b in range(256):
        key = d[:, b].tobytes()
        if key not in cols:
            cols[key] = len(uniq)
            uniq.append(d[:, b])
        byte_class[b] = cols[key]
    nxt = np.stack(uniq, axis=0).astype(np.int32) if uniq else np.zeros((1, d.shape[0]), np.int32)
    return DFA(int(d.shape[0]), int(q0), byte_class, nxt, np.asarray(accept, dtype=np.int32),
               list(kind_names or []))


def dfa_from_edges(n_states: int, edges: Sequence[Tuple[int, int, int]], accept: Dict[int, int],
                   q0: int = 0, kind_names: Optional[List[str]] = None) -> DFA:
    """Hand-assembled automaton from ``(src, byte, dst)`` triples."""
    delta = [[UNDEF] * 256 for _ in range(n_states)]
    for s, b, t in edges:
        delta[s][b] = t
    acc = [accept.get(q, UNDEF) for q in range(n_states)]
    return dfa_from_full_table(delta, acc, q0, kind_names)


def _byte_classes(masks: Sequence[int]) -> List[int]:
    classes = [ALL_BYTES]
    for m in masks:
        nxt = []
        for c in classes:
            a, b = c & m, c & ~m
            if a:
                nxt.append(a)
            if b:
                nxt.append(b)
        classes = nxt
    classes.sort(key=lambda c: (c & -c).bit_length())
    return classes


def compile_tokens(tokens: Sequence[Token], minimize: bool = True) -> DFA:
    """Compile a token list to a (minimised) partial DFA."""
    nfa = _NFA()
    start = nfa.new()
    accept_tag: Dict[int, Tuple[int, int]] = {}
    for kid, tok in enumerate(tokens):
        tree = _Parser(tok.pattern).parse()
        s, e = nfa.build(tree)
        nfa.eps[start].append(s)
        accept_tag[e] = (tok.priority, kid)

    masks = sorted({m for lst in nfa.edges for (m, _) in lst})
    classes = _byte_classes(masks)
    reps = [(c & -c).bit_length() - 1 for c in classes]

    def closure(states) -> frozenset:
        seen = set(states)
        stack = list(states)
        while stack:
            q = stack.pop()
            for t in nfa.eps[q]:
                if t not in seen:
                    seen.add(t)
                    stack.append(t)
        return frozenset(seen)

    d0 = closure([start])
    index = {d0: 0}
    order = [d0]
    trans: List[List[int]] = []
    i = 0
    while i < len(order):
        cur = order[i]
        row = []
        for r in reps:
            moved = [t for q in cur for (m, t) in nfa.edges[q] if (m >> r) & 1]
            if not moved:
                row.append(UNDEF)
                continue
            tgt = closure(moved)
            if tgt not in index:
                index[tgt] = len(order)
                order.append(tgt)
            row.append(index[tgt])
        trans.append(row)
        i += 1

    n = len(order)
    acc = []
    for st in order:
        tags = [accept_tag[q] for q in st if q in accept_tag]
        acc.append(min(tags)[1] if tags else UNDEF)

    n_cls = len(classes)
    if minimize:
        block = {}
        part = []
        for q in range(n):
            part.append(block.setdefault(acc[q], len(block)))
        while True:
            sigs = {}
            new_part = []
            for q in range(n):
                sig = (part[q],) + tuple(part[t] if t != UNDEF else -1 for t in trans[q])
                new_part.append(sigs.setdefault(sig, len(sigs)))
            if len(sigs) == len(set(part)):
                part = new_part
                break
            part = new_part
        # renumber blocks in BFS order from q0 so that the initial state is 0
        rep_of = {}
        for q in range(n):
            rep_of.setdefault(part[q], q)
        bfs = [part[0]]
        seen = {part[0]}
        k = 0
        while k < len(bfs):
            q = rep_of[bfs[k]]
            for t in trans[q]:
                if t != UNDEF and part[t] not in seen:
                    seen.add(part[t])
                    bfs.append(part[t])
            k += 1
        newid = {b: j for j, b in enumerate(bfs)}
        m = len(bfs)
        mtrans = [[UNDEF] * n_cls for _ in range(m)]
        macc = [UNDEF] * m
        for b, j in newid.items():
            q = rep_of[b]
            macc[j] = acc[q]
            for c in range(n_cls):
                t = trans[q][c]
                mtrans[j][c] = newid[part[t]] if t != UNDEF else UNDEF
        trans, acc, n = mtrans, macc, m

    # merge byte classes with identical columns
    col_id: Dict[Tuple[int, ...], int] = {}
    cls_cols: List[Tuple[int, ...]] = []
    remap = []
    for c in range(n_cls):
        col = tuple(trans[q][c] for q in range(n))
        if col not in col_id:
            col_id[col] = len(cls_cols)
            cls_cols.append(col)
        remap.append(col_id[col])
    byte_class = np.zeros(256, dtype=np.uint8)
    for c, cmask in enumerate(classes):
        for b in range(256):
            if (cmask >> b) & 1:
                byte_class[b] = remap[c]
    nxt = np.array(cls_cols, dtype=np.int32).reshape(len(cls_cols), n)
    return DFA(n, 0, byte_class, nxt, np.array(acc, dtype=np.int32), [t.name for t in tokens])
