"""GPU path against the CPU oracle, element by element, through the C ABI.

Bit-exact bar: the (kind, length) stream, its length and con(w) must equal
the oracle's tok(w) (LX_FULL_EXACT) or pi_I(tok(w)) (filtered modes).
"""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu

TILE = 256 * 68
BUF = TILE + 1024


@pytest.fixture(scope="module")
def gpu(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lexlib, lexlib.lx_ctx_create()


_ts_cache = {}


def tokenset(lg, name):
    if name not in _ts_cache:
        _ts_cache[name] = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    return _ts_cache[name]


def gpu_lex(lg, ctx, ts, data, mode, capacity=None, offset=0):
    import torch
    w = np.ascontiguousarray(np.frombuffer(bytes(data), np.uint8) if isinstance(data, (bytes, bytearray)) else data)
    n = int(w.size)
    cap = n + 1 if capacity is None else capacity
    d_raw = torch.empty(n + offset + 16, dtype=torch.uint8, device="cuda")
    if n:
        d_raw[offset:offset + n].copy_(torch.from_numpy(w))
    d_in = d_raw[offset:offset + n] if n else d_raw[:0]
    d_k = torch.zeros(max(cap, 1), dtype=torch.int16, device="cuda")
    d_l = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex(ctx, ts, d_in if n else d_raw, mode, d_k, d_l, n=n, capacity=cap)
    torch.cuda.synchronize()
    m = min(nt, cap)
    k = d_k[:m].cpu().numpy().view(np.uint16)
    l = d_l[:m].cpu().numpy().view(np.uint32)
    return rc, k, l, nt, con


def expected(name, data, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, data)
    if mode != 0:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k, l, con


def check(lg, ctx, name, data, mode, **kw):
    ts = tokenset(lg, name)
    rc, k, l, nt, con = gpu_lex(lg, ctx, ts, data, mode, **kw)
    ek, el, econ = expected(name, data, mode)
    assert rc == 0, lg.lx_strerror(rc)
    assert con == econ, (name, mode, con, econ)
    assert nt == ek.size, (name, mode, nt, ek.size)
    assert np.array_equal(k.astype(np.int64), ek.astype(np.int64)), (name, mode)
    assert np.array_equal(l.astype(np.int64), el.astype(np.int64)), (name, mode)
    return nt


MODES = {"arith": [0, 1, 2], "json": [1, 2], "clike": [1, 2], "clike_row1": [0, 1, 2]}


@pytest.mark.parametrize("name", ["arith", "json", "clike", "clike_row1"])
def test_small_random_inputs(gpu, name):
    lg, ctx = gpu
    wl = {"arith": "arith", "json": "json", "clike": "clike", "clike_row1": "clike"}[name]
    base = bytes(corpus.generate(wl, 1 << 16, seed=21))
    rng = random.Random(3)
    for mode in MODES[name]:
        for _ in range(12):
            a = rng.randrange(0, len(base) - 3000)
            s = bytearray(base[a:a + rng.randint(1, 3000)])
            if rng.random() < 0.4:
                s[rng.randrange(len(s))] = rng.choice(b"\x01`@#$\x7f")
            check(lg, ctx, name, bytes(s), mode)


@pytest.mark.parametrize("n", [0, 1, 2, 15, 16, 17, 67, 68, 69, TILE - 1, TILE, TILE + 1, BUF - 1, BUF, BUF + 1,
                               2 * TILE + 5, 5 * TILE + 3, 9 * TILE + BUF + 7])
def test_ragged_sizes(gpu, n):
    lg, ctx = gpu
    w = corpus.generate("json", 1 << 20, seed=5)[:n]
    check(lg, ctx, "json", w, 2)
    a = corpus.generate("arith", 1 << 20, seed=6)[:n]
    check(lg, ctx, "arith", a, 0)


def test_errors_near_tile_edges(gpu):
    lg, ctx = gpu
    base = corpus.generate("json", 12 * TILE, seed=9).copy()
    for pos in [0, 1, 67, 68, TILE - 1, TILE, TILE + 1, TILE + 1000, BUF - 1, BUF, 3 * TILE - 2, 12 * TILE - 1]:
        w = base.copy()
        w[pos] = ord("#")
        check(lg, ctx, "json", w, 2)
        a = corpus.generate("arith", 12 * TILE, seed=10).copy()
        a[pos] = ord("?")
        check(lg, ctx, "arith", a, 0)


@pytest.mark.parametrize("name,mode,size", [
    ("arith", 0, 1 << 20),          # the 1 MiB exact workload
    ("json", 2, 8 << 20),
    ("json", 1, 1 << 20),           # exact cuts: JSON certifies nothing -> one chunk
    ("clike", 2, 8 << 20),
    ("clike", 1, 1 << 20),
    ("clike_row1", 0, 4 << 20),
])
def test_corpora(gpu, name, mode, size):
    lg, ctx = gpu
    wl = {"clike_row1": "clike"}.get(name, name)
    w = corpus.generate(wl, size)
    check(lg, ctx, name, w, mode)


def test_misaligned_input_pointer(gpu):
    lg, ctx = gpu
    w = corpus.generate("json", 3 * TILE + 99, seed=4)
    for off in (1, 3, 8):
        check(lg, ctx, "json", w, 2, offset=off)


def test_capacity_two_call_protocol(gpu):
    lg, ctx = gpu
    w = corpus.generate("json", 4 * TILE, seed=12)
    ts = tokenset(lg, "json")
    ek, el, econ = expected("json", w, 2)
    cap = ek.size // 3
    rc, k, l, nt, con = gpu_lex(lg, ctx, ts, w, 2, capacity=cap)
    assert rc == lg.LX_E_CAPACITY and nt == ek.size and con == econ
    assert np.array_equal(k.astype(np.int64), ek[:cap]) and np.array_equal(l.astype(np.int64), el[:cap])


def test_full_mode_with_modulo_cuts_is_refused(gpu):
    lg, ctx = gpu
    import torch
    ts = tokenset(lg, "json")
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    k = torch.zeros(16, dtype=torch.int16, device="cuda")
    l = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc, _, _ = lg.lx_lex(ctx, ts, d, 7, k, l)
    assert rc == lg.LX_E_MODE


def test_lex_host_roundtrip(gpu):
    lg, ctx = gpu
    w = corpus.generate("json", 2 * TILE + 77, seed=13)
    ts = tokenset(lg, "json")
    ek, el, econ = expected("json", w, 2)
    hk = np.zeros(w.size + 1, np.uint16)
    hl = np.zeros(w.size + 1, np.uint32)
    rc, nt, con = lg.lx_lex_host(ctx, ts, w, 2, hk, hl)
    assert rc == 0 and nt == ek.size and con == econ
    assert np.array_equal(hk[:nt].astype(np.int64), ek) and np.array_equal(hl[:nt].astype(np.int64), el)


def test_full_size_json_512mib(gpu):
    """The bench workload (512 MiB JSON, filtered modulo) in the bench's launch
    configuration, compared in full with the oracle."""
    lg, ctx = gpu
    w = corpus.generate("json")
    nt = check(lg, ctx, "json", w, 2)
    assert nt > 50_000_000


def test_full_size_clike_512mib(gpu):
    """The 512 MiB C-like workload (filtered modulo I = {ws, line comment},
    cuts at newlines) in the bench's launch configuration, compared in full
    with the oracle."""
    lg, ctx = gpu
    w = corpus.generate("clike")
    assert w.size == 512 << 20
    nt = check(lg, ctx, "clike", w, 2)
    assert nt > 50_000_000


def _dense_lines(rng, n_bytes, min_len, max_len, alphabet):
    """Newline-separated lines of back-to-back short C-like tokens: ranges
    (newline to newline) far longer than a lane's record column."""
    out = bytearray()
    while len(out) < n_bytes:
        ln = rng.randint(min_len, max_len)
        line = bytearray()
        while len(line) < ln:
            line += rng.choice(alphabet)
        out += line[:ln] + b"\n"
    return bytes(out[:n_bytes])


EXPR = [b"a", b"b1", b"x_2", b"+", b"-", b"*", b"/", b"(", b")", b"42", b"0x1f", b" ", b"==", b";", b",", b"if", b"1.5"]


def test_long_ranges_spill(gpu):
    """Ranges of hundreds of kept tokens: compaction plus spill blocks."""
    lg, ctx = gpu
    rng = random.Random(77)
    w = _dense_lines(rng, 3 << 20, 50, 1000, EXPR)
    check(lg, ctx, "clike", w, 2)
    check(lg, ctx, "clike_row1", w, 2)


def test_long_ranges_overflow_fallbacks(gpu):
    """More kept tokens per tile than the stage and the spill region hold
    (one-byte tokens, no separators), and lines longer than the staged halo."""
    lg, ctx = gpu
    rng = random.Random(78)
    dense = _dense_lines(rng, 1 << 20, 900, 1000, [b"+-", b"*", b"%", b"~"])
    check(lg, ctx, "clike", dense, 2)
    long_lines = _dense_lines(rng, 1 << 20, 3000, 9000, EXPR)
    check(lg, ctx, "clike", long_lines, 2)
    check(lg, ctx, "clike", long_lines[: 5 * TILE + 11], 1)


def test_long_ranges_noalloc(gpu):
    """lx_lex_noalloc has no spill region: long ranges take the generic walker."""
    lg, _ = gpu
    import torch
    rng = random.Random(79)
    w = np.frombuffer(_dense_lines(rng, 1 << 20, 50, 1000, EXPR), np.uint8)
    ts = tokenset(lg, "clike")
    d = torch.from_numpy(w.copy()).cuda()
    k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex_noalloc(ts, d, 2, k, l)
    ek, el, econ = expected("clike", w, 2)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)


@pytest.mark.parametrize("kernel", ["warp", "tile"])
@pytest.mark.parametrize("name,size", [("json", 96 << 20), ("clike", 130 << 20)])
def test_lex_host_pieces(gpu, name, size, kernel):
    """Inputs of 64 MiB and more go through lx_lex_host in pieces split at
    certified bytes on the host (copies overlapping the lexing; each piece
    at a 16-byte aligned place with its own output range on the warp-tile
    kernel, in one input and output array on the tile kernel): the stream
    must be the same, including a failure inside a later piece and the
    capacity protocol."""
    import torch
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    if kernel == "tile":
        assert lg.lx_ctx_set_kernel(ctx, lg.LX_KERNEL_TILE) == 0
    ts = tokenset(lg, name)
    w = corpus.generate(name, size, seed=14)
    hk = torch.zeros(size // 2, dtype=torch.int16).pin_memory()
    hl = torch.zeros(size // 2, dtype=torch.int32).pin_memory()
    h_in = torch.from_numpy(w.copy()).pin_memory()
    ek, el, econ = expected(name, w, 2)
    rc, nt, con = lg.lx_lex_host(ctx, ts, h_in, 2, hk, hl)
    assert rc == 0 and nt == ek.size and con == econ
    assert np.array_equal(hk[:nt].numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(hl[:nt].numpy().view(np.uint32).astype(np.int64), el)
    # a lexing error two thirds in
    bad = w.copy()
    bad[size * 2 // 3 + 12345] = 0x01
    fk, fl, fcon = expected(name, bad, 2)
    assert fcon < size
    h_bad = torch.from_numpy(bad).pin_memory()
    rc, nt, con = lg.lx_lex_host(ctx, ts, h_bad, 2, hk, hl)
    assert rc == 0 and con == fcon and nt == fk.size
    assert np.array_equal(hk[:nt].numpy().view(np.uint16).astype(np.int64), fk)
    assert np.array_equal(hl[:nt].numpy().view(np.uint32).astype(np.int64), fl)
    # capacity: the first `cap` tokens and the required count
    cap = ek.size // 3
    rc, nt, con = lg.lx_lex_host(ctx, ts, h_in, 2, hk, hl, capacity=cap)
    assert rc == lg.LX_E_CAPACITY and nt == ek.size and con == econ
    assert np.array_equal(hk[:cap].numpy().view(np.uint16).astype(np.int64), ek[:cap])
