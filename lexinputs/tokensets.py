"""Token sets used by the workloads and by the worked examples of the paper.

Each entry is a list of ``Token`` plus the names of the discarded kinds I.
Kinds are numbered by order of definition (the token ID); a lower
``priority`` wins a same-length tie (Section 3).
"""

from __future__ import annotations

import functools
from typing import Dict, List, Tuple

from .automaton import DFA, Token, compile_tokens, dfa_from_edges


def lit(s: str) -> str:
    """Escape a literal string for the pattern syntax."""
    out = []
    for ch in s:
        if ch.isalnum() or ch == "_":
            out.append(ch)
        else:
            out.append("\\" + ch)
    return "".join(out)


# --- workload token sets -------------------------------------------------------

def arith_tokens() -> List[Token]:
    """Small exact-certificate set: identifiers, integers, single operators,
    '==', parentheses, ';', space runs and a newline token."""
    return [
        Token("ident", "[a-z_][a-z0-9_]*"),
        Token("int", "[0-9]+"),
        Token("plus", lit("+")),
        Token("minus", lit("-")),
        Token("star", lit("*")),
        Token("slash", lit("/")),
        Token("assign", lit("=")),
        Token("eq", lit("==")),
        Token("lparen", lit("(")),
        Token("rparen", lit(")")),
        Token("semi", lit(";")),
        Token("space", " +"),
        Token("newline", "\\n"),
    ]


JSON_STRING = '"([\\x20-\\x21\\x23-\\x5b\\x5d-\\xff]|\\\\(["\\\\/bfnrt]|u[0-9a-fA-F]{4}))*"'
JSON_NUMBER = "-?(0|[1-9][0-9]*)(\\.[0-9]+)?([eE][+\\-]?[0-9]+)?"


def json_tokens() -> List[Token]:
    """RFC 8259 lexical forms over bytes; whitespace runs are tokens."""
    return [
        Token("lbrace", lit("{")),
        Token("rbrace", lit("}")),
        Token("lbracket", lit("[")),
        Token("rbracket", lit("]")),
        Token("colon", lit(":")),
        Token("comma", lit(",")),
        Token("true", "true"),
        Token("false", "false"),
        Token("null", "null"),
        Token("number", JSON_NUMBER),
        Token("string", JSON_STRING),
        Token("ws", "[ \\t\\n\\r]+"),
    ]


C_KEYWORDS = (
    "auto break case char const continue default do double else enum extern float for goto if "
    "int long register return short signed sizeof static struct switch typedef union unsigned "
    "void volatile while"
).split()

C_OPERATORS = (
    "[ ] ( ) { } . -> ++ -- & * + - ~ ! / % << >> < > <= >= == != ^ | && || ? : ; ... = *= /= %= "
    "+= -= <<= >>= &= ^= |= ,"
).split()

C_INT = "[0-9]+|0[xX][0-9a-fA-F]+"
C_EXP = "([eE][+\\-]?[0-9]+)"
C_FLOAT = f"[0-9]+\\.[0-9]*{C_EXP}?|\\.[0-9]+{C_EXP}?|[0-9]+{C_EXP}"


def clike_tokens(block_comments: bool = False) -> List[Token]:
    """C-like token set: 32 keywords over identifiers, decimal/hex integers,
    floats, line-bounded strings and characters with escapes, '//' line
    comments, the 46 multi-byte-maximal operators, and whitespace runs.
    With ``block_comments`` the set also has unrestricted ``/* */`` comments
    and strings that may span lines."""
    toks = [Token("kw_" + k, k, 0) for k in C_KEYWORDS]
    toks.append(Token("ident", "[A-Za-z_][A-Za-z0-9_]*", 1))
    toks.append(Token("int", C_INT, 1))
    toks.append(Token("float", C_FLOAT, 1))
    if block_comments:
        toks.append(Token("string", '"([^"\\\\]|\\\\[\\x00-\\xff])*"', 1))
    else:
        toks.append(Token("string", '"([^"\\\\\\n]|\\\\[^\\n])*"', 1))
    toks.append(Token("char", "'([^'\\\\\\n]|\\\\[^\\n])+'", 1))
    toks.append(Token("line_comment", "//[^\\n]*", 1))
    if block_comments:
        toks.append(Token("block_comment", "/\\*([^*]|\\*+[^*/])*\\*+/", 1))
    for i, op in enumerate(C_OPERATORS):
        toks.append(Token(f"op{i}_{op}", lit(op), 1))
    toks.append(Token("ws", "[ \\t\\r\\n\\v\\f]+", 1))
    return toks


def single_byte_clike_tokens() -> List[Token]:
    """First row of Table 2: identifiers, numbers, whitespace runs, and
    24 operator/punctuation bytes each spelled as a single byte."""
    toks = [Token("ident", "[A-Za-z_][A-Za-z0-9_]*"), Token("number", "[0-9]+"),
            Token("ws", "[ \\t\\n]+")]
    for i, ch in enumerate("+-*/%=<>!&|^~?:;,.()[]{}"):
        toks.append(Token(f"p{i}", lit(ch)))
    return toks


# --- worked examples of the paper ----------------------------------------------

def utf8_tokens() -> List[Token]:
    """One token per UTF-8 encoding form (Section 4, after Definition 2)."""
    c = "[\\x80-\\xbf]"
    return [
        Token("u1", "[\\x00-\\x7f]"),
        Token("u2", "[\\xc2-\\xdf]" + c),
        Token("u3a", "\\xe0[\\xa0-\\xbf]" + c),
        Token("u3b", "[\\xe1-\\xec]" + c + c),
        Token("u3c", "\\xed[\\x80-\\x9f]" + c),
        Token("u3d", "[\\xee-\\xef]" + c + c),
        Token("u4a", "\\xf0[\\x90-\\xbf]" + c + c),
        Token("u4b", "[\\xf1-\\xf3]" + c + c + c),
        Token("u4c", "\\xf4[\\x80-\\x8f]" + c + c),
    ]


def lookahead_tokens() -> List[Token]:
    """Section 9's failed-lookahead example: a, a+b and ;.  On a^n every token
    start reads on to the end looking for b (Theta(n^2) steps unguarded), and
    ';' certifies but never occurs."""
    return [Token("a", "a"), Token("apb", "a+b"), Token("semi", lit(";"))]


def ab_dead_chain() -> DFA:
    """T1 = ab.(empty) beside T2 = b, as the paper's automaton:
    q0 -a-> q2 -b-> q1 (no acceptance reachable), q0 -b-> q3 accepting T2."""
    return dfa_from_edges(4, [(0, ord("a"), 2), (2, ord("b"), 1), (0, ord("b"), 3)], {3: 1},
                          kind_names=["T1", "T2"])


def detached_state() -> DFA:
    """T2 = b with a detached q4 -b-> q5 (q5 accepting, q4 unreachable)."""
    return dfa_from_edges(6, [(0, ord("b"), 3), (4, ord("b"), 5)], {3: 0, 5: 0},
                          kind_names=["T2"])


# --- registry --------------------------------------------------------------------

_SETS: Dict[str, Tuple] = {
    "arith": (arith_tokens, ()),
    "json": (json_tokens, ("ws",)),
    "clike": (lambda: clike_tokens(False), ("ws", "line_comment")),
    "clike_block": (lambda: clike_tokens(True), ("ws", "line_comment", "block_comment")),
    "clike_row1": (single_byte_clike_tokens, ("ws",)),
    "utf8": (utf8_tokens, ()),
    "lookahead": (lookahead_tokens, ()),
}


def token_list(name: str) -> List[Token]:
    return _SETS[name][0]()


def discarded_names(name: str) -> Tuple[str, ...]:
    return tuple(_SETS[name][1])


@functools.lru_cache(maxsize=None)
def tokenset(name: str) -> DFA:
    """Compiled minimised automaton for a registered token set (cached)."""
    return compile_tokens(token_list(name))


def discarded_kinds(name: str) -> List[int]:
    dfa = tokenset(name)
    return [dfa.kind_id(n) for n in discarded_names(name)]


FRAME = 0x1E   # ASCII RECORD SEPARATOR, reserved for framing at the producer (Section 7.1)


def framed(dfa: DFA, frame_byte: int = FRAME) -> DFA:
    """``dfa`` with ``frame_byte`` given a rule of its own: a new kind
    ("frame", numbered n_kinds) of that one byte from q0, and no transition on
    the byte from any other state, so no other token admits it."""
    import numpy as np
    from .automaton import dfa_from_full_table, UNDEF
    d = dfa.delta_full().astype(np.int64)
    n = dfa.n_states
    d[:, frame_byte] = UNDEF
    d[dfa.q0, frame_byte] = n
    d = np.vstack([d, np.full((1, 256), UNDEF, np.int64)])
    acc = list(dfa.accept.tolist()) + [dfa.n_kinds]
    names = list(dfa.kind_names) + ["frame"]
    return dfa_from_full_table(d.tolist(), acc, dfa.q0, names)
