"""Launch configurations of the tile kernel (record column height, CTAs per
SM): every configuration must give the oracle's tokens bit for bit -- small
columns force in-place compaction and spill blocks on every range -- and
lx_autotune must keep one of them."""

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lexlib, lexlib.lx_ctx_create()


def _expected(name, w, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k, l, con


def _lex(lg, ctx, ts, d, mode, n):
    import torch
    k = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rc, nt, con = lg.lx_lex(ctx, ts, d, mode, k, l)
    return rc, k[:nt].cpu().numpy().view(np.uint16), l[:nt].cpu().numpy().view(np.uint32), con


@pytest.mark.parametrize("name", ["json", "clike"])
def test_every_config_is_exact(gpu, name):
    import torch
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    w = corpus.generate(name, 2 << 20, seed=41)
    ek, el, econ = _expected(name, w, 2)
    d = torch.from_numpy(w.copy()).cuda()
    for cls in (0, 1):
        for ks in (16, 24, 36, 40, 64, 96):
            for ctas in (0, 1):
                assert lg.lx_ctx_set_config(ctx, ts, 2, ks, ctas, cls) == 0
                got = lg.lx_ctx_get_config(ctx, ts, 2)
                assert got[:2] == (ks, ctas) and (got[2] == 1 if cls else True)
                rc, k, l, con = _lex(lg, ctx, ts, d, 2, w.size)
                assert rc == 0 and con == econ, (cls, ks, ctas)
                assert np.array_equal(k.astype(np.int64), ek), (cls, ks, ctas)
                assert np.array_equal(l.astype(np.int64), el), (cls, ks, ctas)


def test_invalid_config(gpu):
    lg, ctx = gpu
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    assert lg.lx_ctx_set_config(ctx, ts, 2, 8, 0) == lg.LX_E_INVAL
    assert lg.lx_ctx_set_config(ctx, ts, 2, 200, 0) == lg.LX_E_INVAL
    assert lg.lx_ctx_set_config(ctx, ts, 2, 40, 0, 2) == lg.LX_E_INVAL
    assert lg.lx_ctx_set_config(ctx, ts, 9, 40, 0) == lg.LX_E_MODE


def test_autotune_then_lex(gpu):
    import torch
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    w = corpus.generate("json", 16 << 20, seed=42)
    d = torch.from_numpy(w.copy()).cuda()
    k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
    assert lg.lx_autotune(ctx, ts, 2, d, k, l) == 0
    ks, ctas, cls, ms = lg.lx_ctx_get_config(ctx, ts, 2)
    assert ks in (24, 32, 36, 40, 48, 56, 64) and ms > 0
    ek, el, econ = _expected("json", w, 2)
    rc, kk, ll, con = _lex(lg, ctx, ts, d, 2, w.size)
    assert rc == 0 and con == econ
    assert np.array_equal(kk.astype(np.int64), ek) and np.array_equal(ll.astype(np.int64), el)


def test_batch_uses_config(gpu):
    """A batch after a configuration change (the cached graph is rebuilt)."""
    import torch
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    names = ("json", "clike")
    sets = [lg.lx_compile_tokenset(T.tokenset(n), T.discarded_kinds(n)) for n in names]
    spec = corpus.batch_spec(24, seed=43, median=32 << 10, sigma=1.0, lo=1, hi=256 << 10)
    host, offs = corpus.generate_batch(spec)
    d = torch.from_numpy(host).cuda()
    total = sum(s for _, s, _ in spec)
    k = torch.zeros(total + 64, dtype=torch.int16, device="cuda")
    l = torch.zeros(total + 64, dtype=torch.int32, device="cuda")
    docs = [((d.data_ptr() + o, s), names.index(nm)) for (nm, s, _), o in zip(spec, offs)]
    for ks, cls in ((40, 0), (16, 1)):
        for ts in sets:
            assert lg.lx_ctx_set_config(ctx, ts, 2, ks, 0, cls) == 0
        rc, n_total, res = lg.lx_lex_batch(ctx, sets, docs, 2, k, l)
        assert rc == 0
        kk = k[:n_total].cpu().numpy().view(np.uint16)
        ll = l[:n_total].cpu().numpy().view(np.uint32)
        for (nm, s, _), o, (off, nt, con) in zip(spec, offs, res):
            ek, el, econ = _expected(nm, host[o:o + s], 2)
            assert con == econ and nt == ek.size
            assert np.array_equal(kk[off:off + nt].astype(np.int64), ek)
            assert np.array_equal(ll[off:off + nt].astype(np.int64), el)


def test_default_config_prefers_occupancy(gpu):
    """JSON's byte-indexed table is 18 KB; its class-indexed one fits three
    CTAs per SM, which the default configuration takes."""
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    ks, ctas, cls, ms = lg.lx_ctx_get_config(ctx, ts, 2)
    assert cls == 1 and 32 <= ks <= 40 and ms == 0
    tc = lg.lx_compile_tokenset(T.tokenset("clike"), T.discarded_kinds("clike"))
    assert lg.lx_ctx_get_config(ctx, tc, 2)[:3] == (40, 0, 1)   # class-indexed anyway


def test_wide_class_form_on_gpu(gpu):
    """More than 128 byte classes, both table forms."""
    import random
    import torch
    from test_walk_table_model import wide_class_dfa
    lg, _ = gpu
    ctx = lg.lx_ctx_create()
    dfa, alpha = wide_class_dfa()
    ts = lg.lx_compile_tokenset(dfa, [1])
    rng = random.Random(8)
    w = np.frombuffer(bytes(rng.choice(alpha) for _ in range(300000)), np.uint8)
    d = torch.from_numpy(w.copy()).cuda()
    for mode in (0, 1):
        k, l, con = oracle.lex(dfa, w)
        if mode:
            k, l = oracle.discard(k, l, [1], dfa.n_kinds)
        for cls in (0, 1):
            assert lg.lx_ctx_set_config(ctx, ts, mode, 40, 0, cls) == 0
            rc, kk, ll, c2 = _lex(lg, ctx, ts, d, mode, w.size)
            assert rc == 0 and c2 == con, (mode, cls)
            assert np.array_equal(kk.astype(np.int64), k) and np.array_equal(ll.astype(np.int64), l)
