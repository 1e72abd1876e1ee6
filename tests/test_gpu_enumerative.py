"""lx_lex_enumerative against the oracle, element by element (GPU).

The refused token set (C-like with block comments: no certified byte) on its
corpus, malformed inputs, ragged sizes around the 4096-byte chunk target,
random small automata on long random strings (many chunks, chunk starts with
several candidate contexts, targets without a start), and certified token
sets (the enumeration does not depend on certificates)."""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T
from lexinputs.automaton import Token, compile_tokens

from test_oracle_bruteforce import _random_automata

pytestmark = pytest.mark.gpu
CH = 4096


@pytest.fixture(scope="module")
def gpu(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lexlib, lexlib.lx_ctx_create()


def run(lg, ctx, ts, w, mode, capacity=None):
    import torch
    w = np.ascontiguousarray(np.frombuffer(bytes(w), np.uint8) if isinstance(w, (bytes, bytearray)) else w)
    n = int(w.size)
    cap = n + 1 if capacity is None else capacity
    d = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    if n:
        d[:n].copy_(torch.from_numpy(w))
    k = torch.zeros(max(cap, 1), dtype=torch.int16, device="cuda")
    l = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex_enumerative(ctx, ts, d, mode, k, l, n=n, capacity=cap)
    m = min(nt, cap)
    return rc, k[:m].cpu().numpy().view(np.uint16), l[:m].cpu().numpy().view(np.uint32), nt, con


def check(lg, ctx, dfa, disc, w, mode, ts=None):
    ts = ts or lg.lx_compile_tokenset(dfa, disc)
    rc, k, l, nt, con = run(lg, ctx, ts, w, mode)
    ek, el, econ = oracle.lex(dfa, w)
    if mode != 0:
        ek, el = oracle.discard(ek, el, disc, dfa.n_kinds)
    assert rc == 0, lg.lx_strerror(rc)
    assert con == econ, (con, econ)
    assert nt == ek.size, (nt, ek.size)
    assert np.array_equal(k.astype(np.int64), ek.astype(np.int64))
    assert np.array_equal(l.astype(np.int64), el.astype(np.int64))


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("size", [1 << 20, 8 << 20])
def test_refused_set_corpus(gpu, mode, size):
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    check(lg, ctx, dfa, disc, corpus.generate("clike_block", size), mode)


@pytest.mark.parametrize("n", [0, 1, 2, 255, 256, 257, CH - 1, CH, CH + 1, CH + 255, CH + 256, 2 * CH,
                               7 * CH + 3, 33 * CH + 1000])
def test_ragged_sizes(gpu, n):
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    w = corpus.generate("clike_block", 1 << 18, seed=9)[:n]
    check(lg, ctx, dfa, disc, w, 2)


def test_malformed_inputs(gpu):
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    ts = lg.lx_compile_tokenset(dfa, disc)
    base = corpus.generate("clike_block", 40 * CH, seed=10)
    rng = random.Random(3)
    for pos in [0, 1, CH - 1, CH, CH + 1, 5 * CH + 17, 40 * CH - 1] + [rng.randrange(40 * CH) for _ in range(6)]:
        w = base.copy()
        w[pos] = ord("`")   # in no token, and not inside strings or comments everywhere
        check(lg, ctx, dfa, disc, w, 2, ts=ts)
        check(lg, ctx, dfa, disc, w, 0, ts=ts)


def test_unterminated_block_comment(gpu):
    """A '/*' that never closes: the longest match backtracks to '/' and the
    comment body lexes as ordinary tokens (the comment start is in one chunk,
    its would-be body spans many)."""
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    body = bytes(corpus.generate("clike", 30 * CH, seed=11)).replace(b"*/", b"* /")
    w = b"x = a /* " + body
    check(lg, ctx, dfa, disc, w, 2)
    check(lg, ctx, dfa, disc, w, 0)


def test_random_automata_long_strings(gpu):
    lg, ctx = gpu
    rng = random.Random(12)
    for dfa in _random_automata(505, 12, 12):
        ts = lg.lx_compile_tokenset(dfa, [])
        for n in (3 * CH + 77, 10 * CH):
            w = bytes(rng.choice(b"abc") for _ in range(n))
            check(lg, ctx, dfa, [], w, 0, ts=ts)


def test_long_tokens_across_chunks(gpu):
    """Tokens far longer than a chunk: every chunk start is mid-token."""
    lg, ctx = gpu
    dfa = compile_tokens([Token("as", "a+", 0), Token("b", "b", 0), Token("ws", "[ \\n]+", 0)])
    for w in [b"a" * (9 * CH + 5), (b"a" * 5000 + b" b\n") * 30, b"b" + b"a" * (3 * CH) + b"c"]:
        check(lg, ctx, dfa, [2], w, 0)
        check(lg, ctx, dfa, [2], w, 2)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("name", ["json", "clike", "arith"])
def test_certified_sets_too(gpu, name, mode):
    # JSON and C-like certify no byte exactly: their full stream and their
    # filtered stream under exact cuts go through enumeration
    lg, ctx = gpu
    dfa, disc = T.tokenset(name), T.discarded_kinds(name)
    check(lg, ctx, dfa, disc, corpus.generate(name, 2 << 20, seed=13), mode)


def test_capacity(gpu):
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    ts = lg.lx_compile_tokenset(dfa, disc)
    w = corpus.generate("clike_block", 20 * CH, seed=14)
    ek, el, econ = oracle.lex(dfa, w)
    ek, el = oracle.discard(ek, el, disc, dfa.n_kinds)
    rc, k, l, nt, con = run(lg, ctx, ts, w, 2, capacity=ek.size // 2)
    assert rc == lg.LX_E_CAPACITY and nt == ek.size and con == econ
    assert np.array_equal(k.astype(np.int64), ek[:ek.size // 2]) and np.array_equal(l.astype(np.int64), el[:ek.size // 2])


@pytest.mark.parametrize("off", [1, 3, 8, 15])
def test_unaligned_input(gpu, off):
    # an input that does not start on a 16-byte boundary is read byte by byte
    import torch
    lg, ctx = gpu
    dfa, disc = T.tokenset("clike_block"), T.discarded_kinds("clike_block")
    ts = lg.lx_compile_tokenset(dfa, disc)
    w = corpus.generate("clike_block", 5 * CH + 77, seed=15)
    n = int(w.size)
    d = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
    d[off:off + n].copy_(torch.from_numpy(w.copy()))
    k = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex_enumerative(ctx, ts, d[off:off + n], 0, k, l)
    ek, el, econ = oracle.lex(dfa, w)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)
