"""The failed-lookahead guard (Section 9: over the tokens a, a+b and ; the
input a^n costs Theta(n^2) steps of longest-match scanning, and certified cuts
do not help where the certified byte never occurs), through the C ABI:

* lx_liveness against the oracle's live sets element by element, on inputs
  that span several 4096-byte pieces with a ragged tail, and against the
  closed form on a^n at 10^6 bytes;
* a^n with n = 10^6 and 2 * 10^6 through lx_lex, lx_lex_enumerative and
  lx_lex_speculative: the closed form (n tokens a of length 1, consumed n),
  and the time linear in n;
* (a^k ;)^m: the warp-tile kernel's backtracking runs past its budget inside
  chunks of k bytes and hands the input to the guarded enumerative path;
  element by element against the oracle;
* a token spanning many chunks (a 2 MB block comment; an unterminated JSON
  string) on the enumerative and speculative paths, against the oracle.
"""

import time

import numpy as np
import pytest

import oracle
from oracle import live as L
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    return lg, lg.lx_ctx_create()


_ts = {}


def tokenset(lg, name):
    if name not in _ts:
        _ts[name] = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    return _ts[name]


def member_sets(lg, name, ids):
    rc, blob, m = lg.lx_tokenset_liveness(tokenset(lg, name))
    assert rc == 0
    R, S, W = m["R"], m["S"], m["W"]
    mem = blob[m["member_off"]:m["member_off"] + 4 * R * W].view(np.uint32).reshape(R, W)
    table = np.array([[(int(mem[r][q >> 5]) >> (q & 31)) & 1 for q in range(S)] for r in range(R)], dtype=bool)
    return table[ids]


def dev(w):
    import torch
    w = np.ascontiguousarray(np.frombuffer(bytes(w), np.uint8) if isinstance(w, (bytes, bytearray)) else w)
    d = torch.zeros(w.size + 16, dtype=torch.uint8, device="cuda")
    if w.size:
        d[:w.size].copy_(torch.from_numpy(w.copy()))
    return d[:w.size] if w.size else d[:0], w


def live_ids(lg, ctx, name, w):
    import torch
    d, w = dev(w)
    out = torch.full((w.size + 1,), 0xAB, dtype=torch.uint8, device="cuda")
    rc = lg.lx_liveness(ctx, tokenset(lg, name), d, out, n=w.size)
    assert rc == 0, lg.lx_strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["json", "clike", "clike_block", "lookahead"])
def test_liveness_against_the_oracle(env, name):
    lg, ctx = env
    rng = np.random.default_rng(3)
    if name == "lookahead":
        base = np.frombuffer(bytes(rng.choice(list(b"aaaaaab;"), 20000).astype(np.uint8)), np.uint8)
    else:
        base = corpus.generate(name, 20000, seed=9)
    for n in (0, 1, 17, 4095, 4096, 4097, 3 * 4096 + 77):
        w = base[:n]
        ids = live_ids(lg, ctx, name, w)
        got = member_sets(lg, name, ids)
        want = L.live_sets(T.tokenset(name), w)
        assert np.array_equal(got, want), (name, n)


def test_liveness_closed_form_at_a_million(env):
    lg, ctx = env
    n = 1_000_000
    dfa = T.tokenset("lookahead")
    ids = live_ids(lg, ctx, "lookahead", b"a" * n)
    sets = member_sets(lg, "lookahead", ids)
    q0 = dfa.q0
    assert sets[:n, q0].all() and sets[:n].sum() == n      # live_k = {q0}
    assert not sets[n].any()
    w = b"a" * (n - 1) + b"b"
    sets = member_sets(lg, "lookahead", live_ids(lg, ctx, "lookahead", w))
    d = dfa.delta_full()
    A = int(d[q0, ord("a")])
    B = int(d[A, ord("a")])
    assert sets[:n - 1, q0].all() and sets[:n - 1, A].all() and sets[:n - 1, B].all()
    assert sets[:n - 1].sum() == 3 * (n - 1)


def run(lg, fn, ctx, ts, w, mode, *extra):
    import torch
    d, w = dev(w)
    cap = w.size + 1
    k = torch.zeros(cap, dtype=torch.int16, device="cuda")
    l = torch.zeros(cap, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = fn(ctx, ts, *extra, d, mode, k, l, n=w.size, capacity=cap) if extra else \
        fn(ctx, ts, d, mode, k, l, n=w.size, capacity=cap)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rc, nt, con = res[:3]
    m = min(nt, cap)
    return rc, nt, con, k[:m].cpu().numpy().view(np.uint16).astype(np.int64), \
        l[:m].cpu().numpy().view(np.uint32).astype(np.int64), dt


def spec(lg):
    def f(ctx, ts, model, d, mode, k, l, n, capacity):
        return lg.lx_lex_speculative(ctx, ts, model, d, mode, k, l, n=n, capacity=capacity)
    return f


@pytest.mark.parametrize("path", ["lex", "enumerative", "speculative"])
def test_a_to_the_n_linear(env, path):
    lg, ctx = env
    ts = tokenset(lg, "lookahead")
    dfa = T.tokenset("lookahead")
    ka = dfa.kind_id("a")
    times = []
    for n in (1_000_000, 2_000_000):
        w = b"a" * n
        if path == "lex":
            r = run(lg, lg.lx_lex, ctx, ts, w, 0)
        elif path == "enumerative":
            r = run(lg, lg.lx_lex_enumerative, ctx, ts, w, 0)
        else:
            r = run(lg, spec(lg), ctx, ts, w, 0, None)
        rc, nt, con, k, l, dt = r
        assert rc == 0 and nt == n and con == n, (path, n, rc, nt, con)
        assert (k == ka).all() and (l == 1).all()
        times.append(dt)
    # the second call warms nothing the first did not: linear means about 2x
    assert times[1] < 4.0 * times[0] + 0.05, times


def test_oracle_agrees_on_small_a_to_the_n(env):
    lg, ctx = env
    ts = tokenset(lg, "lookahead")
    for n in (1, 2, 3, 4095, 4096, 4097, 9000):
        w = b"a" * n + b"b" if n % 2 else b"a" * n
        ek, el, econ = oracle.lex(T.tokenset("lookahead"), w)
        for fn in (lg.lx_lex, lg.lx_lex_enumerative):
            rc, nt, con, k, l, _ = run(lg, fn, ctx, ts, w, 0)
            assert rc == 0 and con == econ and np.array_equal(k, ek) and np.array_equal(l, el), (n, fn)


@pytest.mark.parametrize("k", [300, 1000, 3000])
def test_runs_between_cuts(env, k):
    # ';' occurs every k+1 bytes: the warp kernel's chunks hold a^k, whose
    # backtracking is quadratic in k unguarded
    lg, ctx = env
    ts = tokenset(lg, "lookahead")
    m = max(4, 1_000_000 // (k + 1))
    w = (b"a" * k + b";") * m
    ek, el, econ = oracle.lex(T.tokenset("lookahead"), w)
    for fn in (lg.lx_lex, lg.lx_lex_enumerative):
        rc, nt, con, kk, ll, dt = run(lg, fn, ctx, ts, w, 0)
        assert rc == 0 and con == econ and np.array_equal(kk, ek) and np.array_equal(ll, el), (k, fn)
    # with one malformed byte near the end
    w2 = bytearray(w)
    w2[len(w2) - 5] = ord("?")
    ek, el, econ = oracle.lex(T.tokenset("lookahead"), bytes(w2))
    rc, nt, con, kk, ll, dt = run(lg, lg.lx_lex, ctx, ts, bytes(w2), 0)
    assert rc == 0 and con == econ and np.array_equal(kk, ek) and np.array_equal(ll, el)


def expected(name, w, mode):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return k.astype(np.int64), l.astype(np.int64), con


def test_token_spanning_many_chunks(env):
    lg, ctx = env
    ts = tokenset(lg, "clike_block")
    base = corpus.generate("clike_block", 1 << 20, seed=31)
    nl = int(np.flatnonzero(base == 10)[1000]) + 1
    body = np.frombuffer(b"/*" + b"x = y; // not code\n" * 100_000 + b"*/\n", np.uint8)
    w = np.concatenate([base[:nl], body, base[nl:]])
    for mode in (0, 2):
        ek, el, econ = expected("clike_block", w, mode)
        for fn, extra in ((lg.lx_lex_enumerative, ()), (spec(lg), (None,))):
            rc, nt, con, k, l, dt = run(lg, fn, ctx, ts, w, mode, *extra)
            assert rc == 0 and con == econ and np.array_equal(k, ek) and np.array_equal(l, el), (mode, fn)


def test_unterminated_string(env):
    # a quote that never closes: every chunk after it is entered inside the
    # string and would read on to the end of the input
    lg, ctx = env
    ts = tokenset(lg, "json")
    base = corpus.generate("json", 1 << 20, seed=32).copy()
    cut = int(np.flatnonzero(base == 10)[50]) + 1
    w = np.concatenate([base[:cut], np.frombuffer(b'"', np.uint8),
                        np.full(3 << 20, ord("x"), np.uint8)])
    for mode in (0, 1, 2):
        ek, el, econ = expected("json", w, mode)
        for fn in (lg.lx_lex, lg.lx_lex_enumerative):
            rc, nt, con, k, l, dt = run(lg, fn, ctx, ts, w, mode)
            assert rc == 0 and con == econ == cut and np.array_equal(k, ek) and np.array_equal(l, el), (mode, fn)


def test_host_path_hands_over(env):
    # lx_lex_host: a piece whose warp-kernel launch runs past its step budget
    # ((a^k ;)^m) or past the sparse limit (a^n: no certified byte occurs)
    # makes the call lex the whole input through lx_lex's guarded plan
    lg, ctx = env
    ts = tokenset(lg, "lookahead")
    dfa = T.tokenset("lookahead")
    w = (b"a" * 1000 + b";") * 1000
    ek, el, econ = oracle.lex(dfa, w)
    arr = np.frombuffer(w, np.uint8).copy()
    hk = np.zeros(arr.size + 1, np.int16)
    hl = np.zeros(arr.size + 1, np.int32)
    rc, nt, con = lg.lx_lex_host(ctx, ts, arr, 0, hk, hl)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(hk[:nt].view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(hl[:nt].view(np.uint32).astype(np.int64), el)
    n = 1_000_000
    arr = np.full(n, ord("a"), np.uint8)
    hk = np.zeros(n + 1, np.int16)
    hl = np.zeros(n + 1, np.int32)
    t0 = time.perf_counter()
    rc, nt, con = lg.lx_lex_host(ctx, ts, arr, 0, hk, hl)
    assert rc == 0 and nt == n and con == n and time.perf_counter() - t0 < 10.0
    assert (hk[:n] == dfa.kind_id("a")).all() and (hl[:n] == 1).all()
