"""Exhaustive checks of the oracle's certificates on tiny automata.

For every string over a small alphabet up to a length bound, the oracle's
serial scanner is run on the whole string and on the string cut before every
occurrence of a certified byte, and the statements of the paper are checked:

* Lemma 1: in a completely tokenizable string every occurrence of an exactly
  certified byte is a token boundary.
* Theorem 1: cutting at them reproduces tok(w) by ordered concatenation.
* Corollary 1 / Lemma 3: on malformed input the concatenation up to the first
  failing chunk equals tok(w) and the failing chunk halts at con(w).
* Theorem 3: cutting at bytes certified modulo I preserves pi_I(tok(w)); and
  the extension to malformed input adopted by the GPU path (the chunk holding
  the first failure halts at con(w), the pi_I image before it is unchanged).
* Theorem 2 (necessity): for every byte the exact condition rejects, the
  constructive witness w = u b v is completely tokenizable and puts b strictly
  inside its only token.
* Proposition 1 / Corollary 2: a vacuous byte occurs in no completely
  tokenizable string; every certified byte is certified modulo any I
  (Proposition 3, first half).

Automata come from random regular-expression token sets and from random
hand-assembled tables (which have unreachable and dead states, the cases the
live restriction exists for).
"""

import itertools
import random
from collections import deque

import numpy as np

import oracle
from lexinputs.automaton import Token, compile_tokens, dfa_from_edges

ALPHA = b"abc"


def _rand_regex(rng, depth=0):
    r = rng.random()
    if depth > 2 or r < 0.35:
        return rng.choice(["a", "b", "c", "[ab]", "[bc]", "[ac]"])
    if r < 0.55:
        return _rand_regex(rng, depth + 1) + _rand_regex(rng, depth + 1)
    if r < 0.7:
        return "(" + _rand_regex(rng, depth + 1) + "|" + _rand_regex(rng, depth + 1) + ")"
    return "(" + _rand_regex(rng, depth + 1) + ")" + rng.choice(["*", "+", "?"])


def _random_automata(seed, n_regex, n_table):
    rng = random.Random(seed)
    out = []
    for _ in range(n_regex):
        toks = [Token(f"t{i}", _rand_regex(rng), rng.randint(0, 1)) for i in range(rng.randint(1, 4))]
        out.append(compile_tokens(toks))
    for _ in range(n_table):
        S = rng.randint(1, 6)
        edges = [(q, b, rng.randrange(S)) for q in range(S) for b in ALPHA if rng.random() < 0.55]
        acc = {q: rng.randrange(3) for q in range(S) if rng.random() < 0.45}
        out.append(dfa_from_edges(S, edges, acc, q0=0, kind_names=["k0", "k1", "k2"]))
    return out


def _strings(max_len):
    for L in range(1, max_len + 1):
        for t in itertools.product(ALPHA, repeat=L):
            yield bytes(t)


def _boundaries(lens):
    return set(np.concatenate([[0], np.cumsum(lens)]).tolist()) if len(lens) else {0}


def _bfs_path(delta, live, src, targets):
    """Shortest word over delta+ from src into any state of ``targets``."""
    prev = {src: None}
    dq = deque([src])
    while dq:
        q = dq.popleft()
        if q in targets:
            word = []
            while prev[q] is not None:
                q, b = prev[q]
                word.append(b)
            return bytes(reversed(word))
        for b in ALPHA:
            t = int(delta[q, b])
            if t >= 0 and live[q] and live[t] and t not in prev:
                prev[t] = (q, b)
                dq.append(t)
    return None


def _nonempty_cycle(delta, live, q0):
    for b in ALPHA:
        t = int(delta[q0, b])
        if t >= 0 and live[q0] and live[t]:
            rest = _bfs_path(delta, live, t, {q0})
            if rest is not None:
                return bytes([b]) + rest
    return None


def _check_automaton(dfa, max_len, rng):
    a = oracle.Automaton(dfa)
    n_kinds = max(a.n_kinds, 1)
    I = [k for k in range(n_kinds) if rng.random() < 0.5]
    c = oracle.certificates(a, I)
    c0 = oracle.certificates(a, [])
    assert np.array_equal(c0.exact_raw, c0.modulo_raw)            # I = empty set
    assert np.all(~c.exact_raw | c.modulo_raw)                     # Proposition 3
    delta, live, tau = a.delta, c.live, a.tau
    d0_live = np.array([delta[a.q0, b] >= 0 and live[a.q0] and live[delta[a.q0, b]] for b in range(256)])
    assert np.array_equal(c.exact, c.exact_raw & d0_live)          # Corollary 2
    assert np.array_equal(c.modulo, c.modulo_raw & d0_live)        # Proposition 2

    for w in _strings(max_len):
        k, l, con = oracle.lex(a, w)
        complete = con == len(w)
        bounds = _boundaries(l)
        if complete:
            for i, ch in enumerate(w):
                assert not (c.exact_raw[ch] and not d0_live[ch]), "vacuous byte occurred"
                if c.exact_raw[ch]:
                    assert i in bounds, ("Lemma 1", w, i)
        # Theorem 1 / Corollary 1
        cuts = [i for i in range(1, len(w)) if c.exact[w[i]]]
        if cuts:
            k2, l2, con2 = oracle.lex_chunks(a, w, cuts)
            assert con2 == con, ("Cor 1 con", w)
            assert list(k2) == list(k) and list(l2) == list(l), ("Thm 1", w)
        # Theorem 3 (and its malformed-input extension)
        cuts = [i for i in range(1, len(w)) if c.modulo[w[i]]]
        if cuts:
            k2, l2, con2 = oracle.lex_chunks(a, w, cuts)
            assert con2 == con, ("modulo con", w, cuts)
            f1 = oracle.discard(k, l, I, n_kinds)
            f2 = oracle.discard(k2, l2, I, n_kinds)
            assert list(f1[0]) == list(f2[0]) and list(f1[1]) == list(f2[1]), ("Thm 3", w, cuts)

    # Theorem 2: witnesses for every rejected byte of the alphabet
    accepting = {q for q in range(a.n_states) if tau[q] >= 0 and live[q]}
    if live[a.q0]:
        for b in ALPHA:
            if c.exact_raw[b]:
                continue
            witness = None
            for q in range(a.n_states):
                t = int(delta[q, b])
                if q != a.q0 and live[q] and t >= 0 and live[t]:
                    u = _bfs_path(delta, live, a.q0, {q})
                    v = _bfs_path(delta, live, t, accepting)
                    witness = (u, v)
                    break
            if witness is None:
                u = _nonempty_cycle(delta, live, a.q0)
                v = _bfs_path(delta, live, int(delta[a.q0, b]), accepting)
                assert u is not None and d0_live[b]
                witness = (u, v)
            u, v = witness
            w = u + bytes([b]) + v
            k, l, con = oracle.lex(a, w)
            assert con == len(w) and len(l) == 1 and len(u) >= 1, ("Thm 2 witness", w)


def test_bruteforce_regex_token_sets():
    rng = random.Random(7)
    for dfa in _random_automata(2024, 45, 0):
        _check_automaton(dfa, 7, rng)


def test_bruteforce_random_tables():
    rng = random.Random(8)
    for dfa in _random_automata(2025, 0, 70):
        _check_automaton(dfa, 7, rng)


def test_bruteforce_paper_examples_length8():
    rng = random.Random(9)
    sets = [
        [Token("a", "a+"), Token("semi", "c")],
        [Token("a", "a*")],
        [Token("t", "(ab)*c")],
        [Token("abstar", "ab*"), Token("bplus", "b+"), Token("c", "c")],
        [Token("a", "a"), Token("apb", "a+b"), Token("c", "c")],
        [Token("ab", "ab")],
        [Token("ba", "ba")],
    ]
    for toks in sets:
        _check_automaton(compile_tokens(toks), 8, rng)
