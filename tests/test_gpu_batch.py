"""lx_lex_batch against the oracle, document by document, through the C ABI.

Every document of a batch must come out exactly as the serial scan lexes it
alone (pi_I(tok(w)) or tok(w), con(w)), at the output offset the batch
reports; the graph captured on the first call must give the same on a second
call of the same shape with other contents, and a new shape must re-capture.
"""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu

NAMES = ("json", "clike")


@pytest.fixture(scope="module")
def env(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    sets = [lg.lx_compile_tokenset(T.tokenset(n), T.discarded_kinds(n)) for n in NAMES]
    return lg, lg.lx_ctx_create(), sets


def _expected(name, w, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode != 0:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k, l, con


def _run_batch(env, spec, host, offs, mode, shift=0, capacity=None):
    import torch
    lg, ctx, sets = env
    d = torch.from_numpy(np.concatenate([host, np.zeros(64, np.uint8)])).cuda()
    total = sum(s for _, s, _ in spec)
    cap = total + len(spec) + 1 if capacity is None else capacity
    k = torch.zeros(max(cap, 1), dtype=torch.int16, device="cuda")
    l = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    base = d.data_ptr() + shift
    docs = [((base + o, s), NAMES.index(nm)) for (nm, s, _), o in zip(spec, offs)]
    rc, n_total, res = lg.lx_lex_batch(ctx, sets, docs, mode, k, l, capacity=cap)
    torch.cuda.synchronize()
    return rc, n_total, res, k[:min(n_total, cap)].cpu().numpy().view(np.uint16), \
        l[:min(n_total, cap)].cpu().numpy().view(np.uint32)


def _check(spec, host, offs, mode, rc, n_total, res, k, l, shift=0):
    assert rc == 0, rc
    ends = []
    for (nm, size, _), o, (out_off, nt, con) in zip(spec, offs, res):
        w = host[o + shift:o + shift + size]
        ek, el, econ = _expected(nm, w, mode)
        assert con == econ, (nm, size, con, econ)
        assert nt == ek.size, (nm, size, nt, ek.size)
        if size:
            assert np.array_equal(k[out_off:out_off + nt].astype(np.int64), ek), (nm, size)
            assert np.array_equal(l[out_off:out_off + nt].astype(np.int64), el), (nm, size)
            ends.append(out_off + nt)
    assert max(ends, default=0) <= n_total


def _spec(n, seed, median, hi):
    sp = corpus.batch_spec(n, seed=seed, median=median, sigma=1.66, lo=1, hi=hi)
    rng = random.Random(seed)
    sp[rng.randrange(n)] = ("json", 0, 1)            # an empty document
    sp[rng.randrange(n)] = ("clike", 0, 2)
    return sp


def test_batch_mixed_sets(env):
    spec = _spec(96, 11, 6 << 10, 300 << 10)
    host, offs = corpus.generate_batch(spec)
    for mode in (1, 2):
        out = _run_batch(env, spec, host, offs, mode)
        _check(spec, host, offs, mode, *out)


def test_batch_graph_replay_and_malformed_docs(env):
    spec = _spec(64, 12, 4 << 10, 120 << 10)
    host, offs = corpus.generate_batch(spec)
    out = _run_batch(env, spec, host, offs, 2)
    _check(spec, host, offs, 2, *out)
    # same shape, other contents: lexing errors in a few documents
    rng = random.Random(5)
    bad = host.copy()
    for i in rng.sample(range(len(spec)), 8):
        if spec[i][1]:
            bad[offs[i] + rng.randrange(spec[i][1])] = 0x01
    out = _run_batch(env, spec, bad, offs, 2)
    _check(spec, bad, offs, 2, *out)
    # a new shape re-captures
    spec2 = spec[:40]
    out = _run_batch(env, spec2, host, offs[:40], 2)
    _check(spec2, host, offs[:40], 2, *out)


def test_batch_misaligned_documents(env):
    """Documents at odd addresses take the plain-load staging path."""
    spec = _spec(24, 13, 8 << 10, 64 << 10)
    host, offs = corpus.generate_batch(spec, align=1)
    shifted = np.concatenate([np.zeros(3, np.uint8), host])
    out = _run_batch(env, spec, shifted, offs, 2, shift=3)
    _check(spec, shifted, offs, 2, *out, shift=3)


def test_batch_capacity(env):
    spec = _spec(16, 14, 8 << 10, 64 << 10)
    host, offs = corpus.generate_batch(spec)
    rc, n_total, res, _, _ = _run_batch(env, spec, host, offs, 2)
    assert rc == 0
    rc2, n_total2, res2, _, _ = _run_batch(env, spec, host, offs, 2, capacity=n_total // 2)
    lg = env[0]
    assert rc2 == lg.LX_E_CAPACITY and n_total2 == n_total and res2 == res


def test_batch_matches_single_calls(env):
    """The batched stream equals the per-document lx_lex streams."""
    import torch
    lg, ctx, sets = env
    spec = _spec(12, 15, 16 << 10, 256 << 10)
    host, offs = corpus.generate_batch(spec)
    rc, n_total, res, k, l = _run_batch(env, spec, host, offs, 2)
    assert rc == 0
    for (nm, size, _), o, (out_off, nt, con) in zip(spec, offs, res):
        if not size:
            continue
        d = torch.from_numpy(host[o:o + size].copy()).cuda()
        kk = torch.zeros(size + 1, dtype=torch.int16, device="cuda")
        ll = torch.zeros(size + 1, dtype=torch.int32, device="cuda")
        rc1, nt1, con1 = lg.lx_lex(ctx, sets[NAMES.index(nm)], d, 2, kk, ll)
        assert rc1 == 0 and nt1 == nt and con1 == con
        assert np.array_equal(kk[:nt].cpu().numpy().view(np.uint16), k[out_off:out_off + nt])
        assert np.array_equal(ll[:nt].cpu().numpy().view(np.uint32), l[out_off:out_off + nt])


def test_full_size_batch_4096_documents(env):
    """The batched bench workload (4096 documents, ~1.9 GiB, JSON + C-like)
    in the bench's launch configuration, every document compared in full."""
    spec = corpus.batch_spec()
    host, offs = corpus.generate_batch(spec)
    out = _run_batch(env, spec, host, offs, 2, capacity=sum(s for _, s, _ in spec) // 3 + 4096)
    _check(spec, host, offs, 2, *out)
