"""The hybrid plan of lx_lex (Section 9: certified cuts where certified bytes
occur, enumerated entry contexts where they do not), element by element
against the oracle through the C ABI:

* a mode whose cut set is empty (JSON under exact cuts) is lexed by the
  enumerative path, never by one lane walking the whole input;
* an input whose certified bytes are too far apart (minified JSON, or a few
  very long lines) makes the warp-tile kernel stop and hand the input to the
  enumerative path;
* lx_lex_host follows the same plan; with the warp kernel forced, the long
  chunks are walked byte by byte and the output is the same.
"""

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    return lg, ts


def expected(w, mode):
    dfa = T.tokenset("json")
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds("json"), dfa.n_kinds)
    return k.astype(np.int64), l.astype(np.int64), con


def gpu(lg, ctx, ts, w, mode):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(w).copy()).cuda()
    k = torch.zeros(w.size + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size + 1, dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex(ctx, ts, d, mode, k, l)
    return rc, nt, con, k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), \
        l[:nt].cpu().numpy().view(np.uint32).astype(np.int64)


def same(got, want):
    rc, nt, con, k, l = got
    ek, el, econ = want
    return rc == 0 and con == econ and nt == ek.size and np.array_equal(k, ek) and np.array_equal(l, el)


def minified(n, seed):
    w = corpus.generate("json", n, seed=seed).copy()
    for b in b"\n\r\t":
        w[w == b] = ord(" ")
    return w


def test_no_exact_certificate_enumerates(env):
    lg, ts = env
    ctx = lg.lx_ctx_create()
    w = corpus.generate("json", 8 << 20, seed=201)
    for mode in (lg.LX_FULL_EXACT, lg.LX_FILTERED_EXACT):
        assert same(gpu(lg, ctx, ts, w, mode), expected(w, mode))


def test_minified_json_falls_back(env):
    lg, ts = env
    ctx = lg.lx_ctx_create()
    w = minified(8 << 20, 202)
    assert same(gpu(lg, ctx, ts, w, lg.LX_FILTERED_MODULO), expected(w, 2))
    bad = w.copy()
    bad[5_000_001] = 0x01
    assert same(gpu(lg, ctx, ts, bad, lg.LX_FILTERED_MODULO), expected(bad, 2))


def test_few_very_long_lines(env):
    lg, ts = env
    ctx = lg.lx_ctx_create()
    base = corpus.generate("json", 4 << 20, seed=203)
    longline = b'{"blob":"' + b"z" * 300_000 + b'"}\n'
    w = np.frombuffer(base[:1 << 20].tobytes() + longline + base[1 << 20:].tobytes(), np.uint8)
    assert same(gpu(lg, ctx, ts, w, lg.LX_FILTERED_MODULO), expected(w, 2))


def test_forced_warp_kernel_walks_long_chunks(env):
    lg, ts = env
    ctx = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(ctx, lg.LX_KERNEL_WARP) == 0
    w = minified(300_000, 204)
    assert same(gpu(lg, ctx, ts, w, lg.LX_FILTERED_MODULO), expected(w, 2))


def test_lex_host_without_certified_byte(env):
    lg, ts = env
    ctx = lg.lx_ctx_create()
    w = corpus.generate("json", 6 << 20, seed=205)
    k = np.zeros(w.size, np.int16)
    l = np.zeros(w.size, np.int32)
    rc, nt, con = lg.lx_lex_host(ctx, ts, w, lg.LX_FILTERED_EXACT, k, l)
    ek, el, econ = expected(w, 1)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].view(np.uint32).astype(np.int64), el)


def test_lex_host_sparse_cuts_hand_over(env):
    # minified JSON through lx_lex_host: the warp kernel stops at the sparse
    # limit and the call takes the whole input through lx_lex's plan
    lg, ts = env
    ctx = lg.lx_ctx_create()
    w = minified(3 << 20, 206)
    k = np.zeros(w.size + 1, np.int16)
    l = np.zeros(w.size + 1, np.int32)
    rc, nt, con = lg.lx_lex_host(ctx, ts, w, lg.LX_FILTERED_MODULO, k, l)
    ek, el, econ = expected(w, 2)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].view(np.uint32).astype(np.int64), el)
