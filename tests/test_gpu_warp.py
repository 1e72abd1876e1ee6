"""The warp-tile kernel of lx_lex (every warp owns 6144-byte tiles, event
codes in the walk table) against the oracle and against the tile kernel,
element by element, through the C ABI.

Both geometries (sparse: 512-byte halo, 1536 staged tokens; dense: 2048 and
768, the rest of a tile's tokens in the warp's global spill slot) on every
case, and the automatic choice between them on repeated calls.

Cases: every token set and mode on seeded corpora at ragged sizes; lexing
errors near tile and slice edges; lines longer than the halo (the last chunk
of a tile leaves it and is walked byte by byte); inputs with no certified
byte at all; more kept tokens per tile than the shared stage holds (up to
one per byte, dense and sparse tiles in turn, full-mode corpora);
backtracking-heavy inputs; the capacity protocol; empty and one-byte inputs.
"""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu

WT = 6144


@pytest.fixture(scope="module")
def env(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    warp = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(warp, lg.LX_KERNEL_WARP) == 0
    assert lg.lx_ctx_set_warp_geometry(warp, lg.LX_WARP_GEOMETRY_SPARSE) == 0
    tile = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(tile, lg.LX_KERNEL_TILE) == 0
    dense = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(dense, lg.LX_KERNEL_WARP) == 0
    assert lg.lx_ctx_set_warp_geometry(dense, lg.LX_WARP_GEOMETRY_DENSE) == 0
    return lg, warp, tile, dense


_ts = {}


def tokenset(lg, name):
    if name not in _ts:
        _ts[name] = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    return _ts[name]


def run(lg, ctx, name, w, mode, capacity=None):
    import torch
    w = np.ascontiguousarray(np.frombuffer(bytes(w), np.uint8) if isinstance(w, (bytes, bytearray)) else w)
    n = int(w.size)
    cap = n + 1 if capacity is None else capacity
    d = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    if n:
        d[:n].copy_(torch.from_numpy(w.copy()))
    k = torch.zeros(max(cap, 1), dtype=torch.int16, device="cuda")
    l = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex(ctx, tokenset(lg, name), d, mode, k, l, n=n, capacity=cap)
    m = min(nt, cap)
    return rc, nt, con, k[:m].cpu().numpy().view(np.uint16).astype(np.int64), \
        l[:m].cpu().numpy().view(np.uint32).astype(np.int64)


def expected(name, w, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k.astype(np.int64), l.astype(np.int64), con


def check(env, name, w, mode, both=True):
    lg, warp, tile, dense = env
    ek, el, econ = expected(name, w, mode)
    for ctx in (warp, dense):   # both geometries
        rc, nt, con, k, l = run(lg, ctx, name, w, mode)
        assert rc == 0, lg.lx_strerror(rc)
        assert con == econ and nt == ek.size, (name, mode, con, econ, nt, ek.size)
        assert np.array_equal(k, ek) and np.array_equal(l, el), (name, mode)
    if both:
        rc2, nt2, con2, k2, l2 = run(lg, tile, name, w, mode)
        assert rc2 == 0 and nt2 == nt and con2 == con
        assert np.array_equal(k2, k) and np.array_equal(l2, l)
    return nt


SETS = [("arith", 0), ("arith", 1), ("arith", 2), ("json", 1), ("json", 2), ("clike", 1), ("clike", 2),
        ("clike_row1", 0), ("clike_row1", 1), ("clike_row1", 2)]


@pytest.mark.parametrize("name,mode", SETS)
def test_corpora_ragged(env, name, mode):
    gen = "clike" if name == "clike_row1" else name
    base = corpus.generate(gen, 3 << 20, seed=101)
    for n in (1, 15, 16, 17, 127, 128, 129, 191, 192, 193, WT - 1, WT, WT + 1, WT + 495, WT + 496, WT + 497,
              WT + 511, WT + 512, WT + 513, WT + 2031, WT + 2032, WT + 2033, WT + 2048, 3 * WT + 77, 100_003,
              base.size):
        check(env, name, base[:n], mode, both=n == base.size)


@pytest.mark.parametrize("name,mode", [("json", 2), ("clike", 2), ("arith", 0)])
def test_errors_near_edges(env, name, mode):
    base = corpus.generate(name, 64 * WT, seed=102)
    rng = random.Random(7)
    spots = [0, 1, 127, 128, 129, WT - 1, WT, WT + 1, 2 * WT - 3, 5 * WT + 128, 9 * WT + 4095]
    spots += [rng.randrange(base.size) for _ in range(6)]
    for pos in spots:
        w = base.copy()
        w[pos] = 0x01 if name != "arith" else ord("?")
        check(env, name, w, mode, both=False)


def test_lines_longer_than_the_halo(env):
    rng = random.Random(8)
    parts = []
    for _ in range(300):
        if rng.random() < 0.3:
            parts.append(b'{"long":"' + b"y" * rng.randint(900, 9000) + b'"}\n')
        else:
            parts.append(b'{"a":[1,2.5,true],"b":"x"}\n')
    w = b"".join(parts)
    check(env, "json", w, 2)
    check(env, "json", w[:-1] + b"\x01", 2)


def test_no_certified_byte(env):
    # minified JSON (no newline): one chunk from offset 0, walked byte by byte
    w = corpus.generate("json", 200_000, seed=103).copy()
    w[w == ord("\n")] = ord(" ")
    w[w == ord("\r")] = ord(" ")
    w[w == ord("\t")] = ord(" ")
    check(env, "json", w, 2)


def test_dense_tokens_overflow_the_stage(env):
    # one-byte tokens: over 1536 kept tokens per 6144-byte tile
    rng = random.Random(9)
    line = lambda: bytes(rng.choice(b"+-*/%~!;,") for _ in range(rng.randint(30, 300))) + b"\n"
    w = b"".join(line() for _ in range(3000))
    check(env, "clike", w, 2)
    check(env, "clike", w, 1, both=False)


def test_every_byte_a_token(env):
    # up to one kept token per byte: a tile's first 1536 go to the shared
    # stage, the rest to the warp's spill slot
    rng = random.Random(11)
    ops = b"()+-*/;"
    w = bytes(rng.choice(ops) for _ in range(20 * WT + 777))
    check(env, "arith", w, 0)
    # dense and sparse tiles in turn: a deferred tile's spill slot is copied
    # out before the warp's next tile fills it
    parts = []
    for i in range(40):
        if i % 3 == 0:
            parts.append(bytes(rng.choice(ops) for _ in range(WT + rng.randint(-500, 500))))
        else:
            parts.append(b"\n".join(b"abc" * rng.randint(1, 40) for _ in range(60)))
    w = b"".join(parts)
    for mode in (0, 2):
        check(env, "arith", w, mode)
    # full-mode C-like and JSON: about 1 850 / 1 400 kept tokens per tile
    for name, seed in (("clike", 105), ("json", 106)):
        check(env, name, corpus.generate(name, (2 << 20) + 4099, seed=seed), 0)


def test_backtracking(env):
    rng = random.Random(10)
    parts = [b"a..b", b"0x", b"x...y", b"1.", b".5", b"a->b", b"a-->b", b" ", b"\n", b";", b"1e+", b"1e5"]
    w = b"".join(rng.choice(parts) for _ in range(200_000))
    check(env, "clike", w, 2)
    w = b"".join(rng.choice([b"===", b"=", b"==", b"a", b"\n", b"(", b" "]) for _ in range(200_000))
    check(env, "arith", w, 0)


def test_capacity_and_small(env):
    lg, warp, tile, dense = env
    w = corpus.generate("json", 300_000, seed=104)
    ek, el, econ = expected("json", w, 2)
    cap = ek.size // 3
    for ctx in (warp, dense):
        rc, nt, con, k, l = run(lg, ctx, "json", w, 2, capacity=cap)
        assert rc == lg.LX_E_CAPACITY and nt == ek.size and con == econ
        assert np.array_equal(k, ek[:cap]) and np.array_equal(l, el[:cap])
    for w in (b"", b"{", b"\n", b"1", b"\x01", b"[1]\n"):
        check(env, "json", w, 2)


def test_warp_kernel_needs_aligned_input(env):
    import torch
    lg, warp, tile, dense = env
    w = corpus.generate("json", 10_000, seed=105)
    d = torch.zeros(w.size + 32, dtype=torch.uint8, device="cuda")
    d[3:3 + w.size].copy_(torch.from_numpy(w.copy()))
    k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
    rc, _, _ = lg.lx_lex(warp, tokenset(lg, "json"), d[3:3 + w.size], 2, k, l)
    assert rc == lg.LX_E_INVAL          # asked for the warp kernel, which needs 16-byte alignment
    auto = lg.lx_ctx_create()
    rc, nt, con = lg.lx_lex(auto, tokenset(lg, "json"), d[3:3 + w.size], 2, k, l)
    ek, el, econ = expected("json", w, 2)
    assert rc == 0 and nt == ek.size and con == econ     # the tile kernel serves it


def test_geometry_setting_and_auto(env):
    lg = env[0]
    assert lg.lx_ctx_set_warp_geometry(lg.lx_ctx_create(), 3) == lg.LX_E_INVAL
    assert lg.lx_ctx_set_warp_geometry(lg.lx_ctx_create(), -1) == lg.LX_E_INVAL
    # AUTO: the first call sparse, later ones as the previous call showed; the
    # stream never changes.  Full-mode C-like (about 1 850 kept tokens per
    # tile) and lines longer than the sparse halo both turn it dense.
    auto = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(auto, lg.LX_KERNEL_WARP) == 0
    rng = random.Random(12)
    long_lines = b"".join(b'{"s":"' + b"z" * rng.randint(600, 1500) + b'"}\n' if rng.random() < 0.2
                          else b'{"a":1}\n' for _ in range(2000))
    for name, w, mode in (("clike", corpus.generate("clike", (1 << 20) + 5, seed=106), 0),
                          ("json", corpus.generate("json", (1 << 20) + 3, seed=107), 2),
                          ("clike", long_lines, 2)):
        ek, el, econ = expected(name, w, mode)
        for _ in range(3):
            rc, nt, con, k, l = run(lg, auto, name, w, mode)
            assert rc == 0 and con == econ and np.array_equal(k, ek) and np.array_equal(l, el)


def test_output_alignment(env):
    # the output arrays at offsets 1-4 elements: tokens are written in groups
    # of 2 (sparse) or 4 (dense) where the arrays are aligned for it, one by
    # one otherwise
    import torch
    lg, warp, tile, dense = env
    for name, mode in (("json", 2), ("clike", 0)):
        w = corpus.generate(name, 3 * WT * 7 + 333, seed=108)
        ek, el, econ = expected(name, w, mode)
        d = torch.from_numpy(w.copy()).cuda()
        for ctx in (warp, dense):
            for off in (1, 2, 3, 4):
                k = torch.zeros(ek.size + 8, dtype=torch.int16, device="cuda")
                l = torch.zeros(ek.size + 8, dtype=torch.int32, device="cuda")
                rc, nt, con = lg.lx_lex(ctx, tokenset(lg, name), d, mode, k[off:], l[off:], capacity=ek.size + 8 - off)
                assert rc == 0 and nt == ek.size and con == econ
                assert np.array_equal(k[off:off + nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
                assert np.array_equal(l[off:off + nt].cpu().numpy().view(np.uint32).astype(np.int64), el)
                assert not k[:off].any() and not l[:off].any() and not k[off + nt:].any()


def test_host_pieces_both_geometries(env):
    # full-mode C-like through lx_lex_host in pieces: the first call sparse,
    # the next dense (about 1 850 kept tokens per tile), both the oracle's
    lg = env[0]
    ctx = lg.lx_ctx_create()
    w = corpus.generate("clike", (70 << 20) + 13, seed=109)
    ek, el, econ = expected("clike", w, 0)
    for _ in range(2):
        hk = np.zeros(ek.size + 1, np.int16)
        hl = np.zeros(ek.size + 1, np.int32)
        rc, nt, con = lg.lx_lex_host(ctx, tokenset(lg, "clike"), w, 0, hk, hl)
        assert rc == 0 and con == econ and nt == ek.size
        assert np.array_equal(hk[:nt].view(np.uint16).astype(np.int64), ek)
        assert np.array_equal(hl[:nt].view(np.uint32).astype(np.int64), el)
