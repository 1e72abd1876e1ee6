"""The one-launch batch (every document of every token set in one launch of
the warp-tile kernel, the sets' class-form tables side by side in shared
memory), the async lx_lex and the warps-per-CTA setting, through the C ABI:

* one-launch batches against the oracle document by document, and against
  the per-set tile-kernel batches (LX_KERNEL_TILE), on mixed JSON / C-like
  and JSON / block-comment C-like batches with empty documents, lexing
  errors and documents shorter than one tile; documents with more kept
  tokens per tile than the shared stage holds; the output in document order;
* lx_lex_async: many launches back to back on one stream, one
  synchronization, every record and stream equal to lx_lex's; the capacity
  status; the argument errors;
* lx_ctx_set_warps: the same tokens at 1, 4, 9 and 20 warps per CTA.
"""

import random

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
    return lexlib


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


def make_batch(names, n, seed, errors=0):
    rng = random.Random(seed)
    spec = corpus.batch_spec(n, seed=seed, median=12 << 10, sigma=1.66, lo=1, hi=400 << 10, names=names)
    spec[rng.randrange(n)] = (names[0], 0, 1)           # empty documents
    spec[rng.randrange(n)] = (names[-1], 0, 2)
    spec[rng.randrange(n)] = (names[0], 5, 3)           # shorter than a word
    host, offs = corpus.generate_batch(spec)
    for _ in range(errors):                             # malformed bytes
        i = rng.randrange(n)
        if spec[i][1] > 10:
            host[offs[i] + rng.randrange(spec[i][1])] = 0x01
    return spec, host, offs


def run_batch(lg, ctx, names, spec, host, offs, mode):
    import torch
    sets = [tokenset(lg, nm) for nm in names]
    d = torch.from_numpy(np.concatenate([host, np.zeros(64, np.uint8)])).cuda()
    cap = sum(s for _, s, _ in spec) + len(spec) + 1
    k = torch.zeros(cap, dtype=torch.int16, device="cuda")
    l = torch.zeros(cap, dtype=torch.int32, device="cuda")
    docs = [((d.data_ptr() + o, s), names.index(nm)) for (nm, s, _), o in zip(spec, offs)]
    rc, n_total, res = lg.lx_lex_batch(ctx, sets, docs, mode, k, l, capacity=cap)
    torch.cuda.synchronize()
    m = min(n_total, cap)
    return rc, n_total, res, k[:m].cpu().numpy().view(np.uint16).astype(np.int64), \
        l[:m].cpu().numpy().view(np.uint32).astype(np.int64)


def check_docs(spec, host, offs, mode, res, k, l):
    for (nm, size, _), o, (out_off, nt, con) in zip(spec, offs, res):
        w = host[o:o + size]
        ek, el, econ = expected(nm, w, mode)
        assert con == econ and nt == ek.size, (nm, size, con, econ, nt, ek.size)
        assert np.array_equal(k[out_off:out_off + nt], ek) and np.array_equal(l[out_off:out_off + nt], el)


@pytest.mark.parametrize("names", [("json", "clike"), ("json", "clike_block")])
def test_one_launch_batch_against_the_oracle(env, names):
    lg = env
    spec, host, offs = make_batch(names, 80, 21, errors=5)
    warp = lg.lx_ctx_create()
    tile = lg.lx_ctx_create()
    assert lg.lx_ctx_set_kernel(tile, lg.LX_KERNEL_TILE) == 0
    for mode in (1, 2):
        rc, n_total, res, k, l = run_batch(lg, warp, names, spec, host, offs, mode)
        assert rc == 0, lg.lx_strerror(rc)
        check_docs(spec, host, offs, mode, res, k, l)
        rc2, n2, res2, k2, l2 = run_batch(lg, tile, names, spec, host, offs, mode)
        assert rc2 == 0
        check_docs(spec, host, offs, mode, res2, k2, l2)
        # the one-launch batch keeps document order: non-empty documents' ranges ascend (in the
        # exact modes the tables carry split-window rows, which keep a batch on the per-set kernels)
        if mode == 2:
            starts = [r[0] for (nm, s, _), r in zip(spec, res) if s]
            assert starts == sorted(starts)
        # a second call of the same shape replays the graph with the same result
        rc3, n3, res3, k3, l3 = run_batch(lg, warp, names, spec, host, offs, mode)
        assert rc3 == 0 and res3 == res and np.array_equal(k3, k)


def test_one_launch_batch_dense_documents(env):
    # C-like documents of one-byte operator tokens (over 1536 kept tokens
    # per tile: the stage spills) between JSON documents, in one launch
    lg = env
    rng = random.Random(12)
    names = ("json", "clike")
    ops = b"+-*%~!;,"
    spec, chunks, offs, pos = [], [], [], 0
    for i in range(30):
        if i % 2:
            lines = rng.randint(1, 400)
            w = b"\n".join(bytes(rng.choice(ops) for _ in range(rng.randint(30, 300))) for _ in range(lines))
            spec.append(("clike", len(w), 0))
        else:
            w = bytes(corpus.generate("json", rng.choice([0, 1000, 50_000]), seed=300 + i))
            spec.append(("json", len(w), 0))
        offs.append(pos)
        chunks.append(w + bytes(-len(w) % 16))
        pos += len(chunks[-1])
    host = np.frombuffer(b"".join(chunks) or b"\0", np.uint8).copy()
    ctx = lg.lx_ctx_create()
    rc, n_total, res, k, l = run_batch(lg, ctx, names, spec, host, offs, 2)
    assert rc == 0, lg.lx_strerror(rc)
    check_docs(spec, host, offs, 2, res, k, l)
    starts = [r[0] for (nm, s, _), r in zip(spec, res) if s]
    assert starts == sorted(starts)


def test_one_launch_batch_tiny_and_single_set(env):
    lg = env
    ctx = lg.lx_ctx_create()
    for n in (1, 2, 7):
        spec, host, offs = make_batch(("json",), n + 3, 40 + n)
        rc, n_total, res, k, l = run_batch(lg, ctx, ("json",), spec, host, offs, 2)
        assert rc == 0
        check_docs(spec, host, offs, 2, res, k, l)


def test_async_back_to_back(env):
    import torch
    lg = env
    ctx = lg.lx_ctx_create()
    ref = lg.lx_ctx_create()
    stream = torch.cuda.Stream()
    rng = random.Random(5)
    jobs = []
    for i in range(48):
        nm = ("json", "clike")[i % 2]
        size = rng.choice([1, 100, 4096, 5000, 70_000, 300_000])
        w = corpus.generate(nm, size, seed=100 + i).copy()
        if i % 7 == 3:
            w[rng.randrange(size)] = 0x01
        jobs.append((nm, w))
    bufs = []
    with torch.cuda.stream(stream):
        for nm, w in jobs:
            d = torch.from_numpy(w).cuda()
            k = torch.zeros(w.size + 1, dtype=torch.int16, device="cuda")
            l = torch.zeros(w.size + 1, dtype=torch.int32, device="cuda")
            r = torch.zeros(24, dtype=torch.uint8, device="cuda")
            rc = lg.lx_lex_async(ctx, tokenset(lg, nm), d, 2, k, l, r, stream=stream)
            assert rc == 0, lg.lx_strerror(rc)
            bufs.append((d, k, l, r))
    stream.synchronize()
    for (nm, w), (d, k, l, r) in zip(jobs, bufs):
        st, nt, con = lg.async_result(r.cpu().numpy())
        k2 = torch.zeros(w.size + 1, dtype=torch.int16, device="cuda")
        l2 = torch.zeros(w.size + 1, dtype=torch.int32, device="cuda")
        rc2, nt2, con2 = lg.lx_lex(ref, tokenset(lg, nm), d, 2, k2, l2)
        assert st == 0 and rc2 == 0 and (nt, con) == (nt2, con2)
        assert torch.equal(k[:nt], k2[:nt]) and torch.equal(l[:nt], l2[:nt])
    # capacity: the record says so and the count is the full one
    w = corpus.generate("json", 50_000, seed=7)
    d = torch.from_numpy(w.copy()).cuda()
    k = torch.zeros(10, dtype=torch.int16, device="cuda")
    l = torch.zeros(10, dtype=torch.int32, device="cuda")
    r = torch.zeros(24, dtype=torch.uint8, device="cuda")
    assert lg.lx_lex_async(ctx, tokenset(lg, "json"), d, 2, k, l, r, capacity=10) == 0
    torch.cuda.synchronize()
    st, nt, con = lg.async_result(r.cpu().numpy())
    ek, el, econ = expected("json", w, 2)
    assert st == lg.LX_E_CAPACITY and nt == ek.size and con == econ
    assert np.array_equal(k.cpu().numpy().view(np.uint16).astype(np.int64), ek[:10])
    # an unaligned input is refused at once
    assert lg.lx_lex_async(ctx, tokenset(lg, "json"), d[1:], 2, k, l, r, capacity=10) == lg.LX_E_INVAL


def test_warps_per_cta(env):
    import torch
    lg = env
    w = corpus.generate("clike", 3 << 20, seed=8)
    d = torch.from_numpy(w.copy()).cuda()
    ek, el, econ = expected("clike", w, 2)
    for nw in (1, 4, 9, 20, 0):
        ctx = lg.lx_ctx_create()
        assert lg.lx_ctx_set_warps(ctx, nw) == 0
        k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
        l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
        rc, nt, con = lg.lx_lex(ctx, tokenset(lg, "clike"), d, 2, k, l)
        assert rc == 0 and con == econ and nt == ek.size
        assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
        assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)
    assert lg.lx_ctx_set_warps(lg.lx_ctx_create(), 21) == lg.LX_E_INVAL
