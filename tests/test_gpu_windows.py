"""Split windows on the GPU: in the exact modes, token sets that certify no
single byte (JSON, C-like) are cut by the warp-tile kernel at certified
two-byte windows (lx_window_certificates); element by element against the
oracle through the C ABI, with the kernel forced and on the default route:
ragged sizes across tiles and slices, malformed bytes, lines longer than the
halo, a 512 MiB JSON corpus under LX_FILTERED_EXACT."""

import random

import numpy as np
import pytest

import oracle
from oracle import windows as W
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
    return lg, warp, lg.lx_ctx_create()


_ts = {}


def tokenset(lg, name):
    if name not in _ts:
        _ts[name] = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    return _ts[name]


def expected(name, w, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k.astype(np.int64), l.astype(np.int64), con


def run(lg, ctx, name, w, mode):
    import torch
    w = np.ascontiguousarray(np.frombuffer(bytes(w), np.uint8) if isinstance(w, (bytes, bytearray)) else w)
    n = int(w.size)
    d = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    if n:
        d[:n].copy_(torch.from_numpy(w.copy()))
    k = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex(ctx, tokenset(lg, name), d[:max(n, 1)] if n else d[:0], mode, k, l, n=n, capacity=n + 1)
    m = min(nt, n + 1)
    return rc, nt, con, k[:m].cpu().numpy().view(np.uint16).astype(np.int64), \
        l[:m].cpu().numpy().view(np.uint32).astype(np.int64)


def check(env, name, w, mode):
    lg, warp, auto = env
    ek, el, econ = expected(name, w, mode)
    for ctx in (warp, auto):
        rc, nt, con, k, l = run(lg, ctx, name, w, mode)
        assert rc == 0, lg.lx_strerror(rc)
        assert con == econ and nt == ek.size, (name, mode, con, econ, nt, ek.size)
        assert np.array_equal(k, ek) and np.array_equal(l, el), (name, mode)


@pytest.mark.parametrize("name,mode", [("json", 0), ("json", 1), ("clike", 0), ("clike", 1)])
def test_window_cuts_ragged(env, name, mode):
    lg = env[0]
    rc, blob, meta = lg.lx_tokenset_walk_table(tokenset(lg, name), mode)
    assert rc == 0 and meta["n_ctx"] > 0
    base = corpus.generate(name, 3 << 20, seed=201)
    # the corpus really has window cuts, and no single certified byte
    assert not oracle.certificates(T.tokenset(name)).exact.any()
    assert len(W.window_cuts(T.tokenset(name), base[:20000])) > 100
    for n in (1, 2, 191, 192, 193, WT - 1, WT, WT + 1, 3 * WT + 77, 100_003, base.size):
        check(env, name, base[:n], mode)


@pytest.mark.parametrize("name,mode", [("json", 1), ("clike", 0)])
def test_window_cuts_malformed(env, name, mode):
    base = corpus.generate(name, 64 * WT, seed=202)
    rng = random.Random(3)
    for pos in [0, 1, 127, 128, WT - 1, WT, WT + 1, 5 * WT + 128] + [rng.randrange(base.size) for _ in range(5)]:
        w = base.copy()
        w[pos] = 0x01
        check(env, name, w, mode)


def test_window_cuts_long_lines(env):
    rng = random.Random(8)
    parts = []
    for _ in range(300):
        if rng.random() < 0.3:
            parts.append(b'{"long":"' + b"y" * rng.randint(900, 9000) + b'"}\n')
        else:
            parts.append(b'{"a":[1,2.5,true],"b":"x"}\n')
    w = b"".join(parts)
    check(env, "json", w, 1)
    check(env, "json", w, 0)


def test_full_size_json_exact_filtered(env):
    """The 512 MiB JSON corpus under LX_FILTERED_EXACT (window cuts), the
    whole stream against the oracle."""
    lg, warp, auto = env
    w = corpus.generate("json", 512 << 20)
    ek, el, econ = expected("json", w, 1)
    rc, nt, con, k, l = run(lg, auto, "json", w, 1)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k, ek) and np.array_equal(l, el)
