"""Speculative lexing of a refused token set and its entry-context model (GPU).

* lx_chunk_contexts labels equal the oracle's context() at every chunk start;
* model windows, the BF16-weight forward and gradient equal the FP64
  reference (oracle/model.py, at the BF16-rounded weights) within FP32
  tolerances, block by block; AdamW steps lower the loss;
* lx_lex_speculative equals the serial oracle bit for bit with no model, a
  random model and a trained one (predictions only change the rescans), on
  the refused C-like corpus, malformed and ragged inputs.
"""

import random

import numpy as np
import pytest

import oracle
from oracle import contexts as OC
from oracle import model as OM
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu
NAME = "clike_block"


@pytest.fixture(scope="module")
def env(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    ts = lg.lx_compile_tokenset(T.tokenset(NAME), T.discarded_kinds(NAME))
    S = lg.lx_tokenset_scan_table(ts)[2]["S"]
    return lg, lg.lx_ctx_create(), ts, S


def _dev(w):
    import torch
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint8).copy()).cuda()


def test_chunk_contexts_match_oracle(env):
    lg, ctx, ts, S = env
    w = corpus.generate(NAME, 1 << 20, seed=51)
    rc, starts, cx = lg.lx_chunk_contexts(ctx, ts, _dev(w))
    assert rc == 0
    ref = OC.contexts(T.tokenset(NAME), w)
    starts = starts.cpu().numpy()
    cx = cx.cpu().numpy().view(np.uint16)
    seen = 0
    for p, c in zip(starts, cx):
        if p < 0:
            continue
        want = ref[p]
        assert (c == lg.CTX_BOUNDARY) == (want == OC.BOUNDARY), p
        if want != OC.BOUNDARY:
            assert c == want, (p, c, want)
        seen += 1
    assert seen > 200


def test_model_forward_and_gradient_match_reference(env):
    import torch
    lg, ctx, ts, S = env
    C = S + 1
    m = lg.Model(C, hidden=32, seed=7)
    w = corpus.generate(NAME, 1 << 18, seed=52)
    rng = np.random.default_rng(3)
    pos = np.sort(rng.integers(0, w.size, size=96)).astype(np.int64)
    pos[:2] = [0, w.size - 1]
    d = _dev(w)
    win = m.windows(d, torch.from_numpy(pos).cuda())
    ref_win = OM.windows(w, pos)
    assert np.array_equal(win.cpu().numpy().astype(np.int64) & 0xFFFF, ref_win)
    # the device computes with BF16 weights and FP32 activations and sums:
    # against the FP64 reference at the BF16-rounded weights only FP32
    # rounding remains
    p = OM.to_bf16(m.get_params().astype(np.float64))
    z = m.forward(win).cpu().numpy()
    rz, _ = OM.forward(p, ref_win, 32, C)
    assert np.max(np.abs(z - rz)) < 1e-4 * (1 + np.max(np.abs(rz)))
    y = rng.integers(0, C, size=pos.size)
    g, loss = m.gradient(win, torch.from_numpy(y.astype(np.int16)).cuda())
    rl, rg = OM.loss_and_grad(p, ref_win, y, 32, C)
    assert abs(loss - rl) < 1e-4 * (1 + abs(rl))
    blocks = np.cumsum([0] + OM.sizes(32, C))
    for lo, hi in zip(blocks[:-1], blocks[1:]):   # every parameter block
        assert np.max(np.abs(g[lo:hi] - rg[lo:hi])) < 1e-5 + 1e-3 * np.max(np.abs(rg[lo:hi])), (lo, hi)
    # and the BF16 weights are the round-to-nearest-even of the FP32 ones
    assert m.n_params == OM.n_params(32, C)


def test_training_lowers_the_loss(env):
    import torch
    lg, ctx, ts, S = env
    m = lg.Model(S + 1, hidden=32, seed=8)
    d = _dev(corpus.generate(NAME, 16 << 20, seed=53))
    W, Y = lg.context_training_set(ctx, ts, m, d)
    assert W.shape[0] > 3000
    first = None
    for it in range(150):
        idx = torch.randint(0, W.shape[0], (256,), device=W.device)
        loss = m.train_step(W[idx].contiguous(), Y[idx].contiguous(), 3e-3)
        first = loss if first is None else first
    _, last = m.gradient(W[:1024].contiguous(), Y[:1024].contiguous())
    assert last < 0.5 * first, (first, last)


def _check(lg, ctx, ts, model, w, mode):
    import torch
    d = _dev(w)
    n = int(w.size)
    k = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rc, nt, con, st = lg.lx_lex_speculative(ctx, ts, model, d, mode, k, l)
    dfa = T.tokenset(NAME)
    ek, el, econ = oracle.lex(dfa, w)
    if mode:
        ek, el = oracle.discard(ek, el, T.discarded_kinds(NAME), dfa.n_kinds)
    assert rc == 0 and con == econ and nt == ek.size, (rc, con, econ, nt, ek.size)
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)
    assert st["rounds"] >= 1
    return st


@pytest.fixture(scope="module")
def trained(env):
    lg, ctx, ts, S = env
    samples = [_dev(corpus.generate(NAME, 32 << 20, seed=s)) for s in (61, 62)]
    return lg.train_context_model(ctx, ts, samples, hidden=64, epochs=3)


@pytest.mark.parametrize("which", ["none", "random", "trained"])
@pytest.mark.parametrize("mode", [0, 2])
def test_speculative_exact(env, trained, which, mode):
    lg, ctx, ts, S = env
    model = {"none": None, "random": lg.Model(S + 1, hidden=16, seed=9), "trained": trained}[which]
    st = _check(lg, ctx, ts, model, corpus.generate(NAME, 8 << 20, seed=54), mode)
    if which == "trained":
        assert st["rescanned"] < 0.2 * st["chunks"], st


def test_trained_model_gains(env, trained):
    # what the network buys: fewer chunks scanned twice than with BOUNDARY
    # guesses (no model) or an untrained network, same exact output
    lg, ctx, ts, S = env
    w = corpus.generate(NAME, 8 << 20, seed=57)
    st_none = _check(lg, ctx, ts, None, w, 0)
    st_rand = _check(lg, ctx, ts, lg.Model(S + 1, hidden=16, seed=10), w, 0)
    st_tr = _check(lg, ctx, ts, trained, w, 0)
    assert st_tr["rescanned"] * 3 < st_none["rescanned"], (st_tr, st_none)
    assert st_tr["rescanned"] * 3 < st_rand["rescanned"], (st_tr, st_rand)
    assert st_tr["rounds"] <= st_none["rounds"]


def test_speculative_malformed_and_ragged(env, trained):
    lg, ctx, ts, S = env
    base = corpus.generate(NAME, 64 * 4096, seed=55)
    rng = random.Random(4)
    for n in [1, 4095, 4096, 4097, 9000, 64 * 4096]:
        _check(lg, ctx, ts, trained, base[:n], 2)
    for pos in [0, 4096, 77777] + [rng.randrange(base.size) for _ in range(3)]:
        w = base.copy()
        w[pos] = ord("`")
        _check(lg, ctx, ts, trained, w, 0)
        _check(lg, ctx, ts, None, w, 2)


@pytest.mark.parametrize("off", [1, 7, 12])
def test_speculative_unaligned_input(env, trained, off):
    # an input that does not start on a 16-byte boundary is read byte by byte
    import torch
    lg, ctx, ts, S = env
    w = corpus.generate(NAME, 3 * 4096 + 1234, seed=58)
    n = int(w.size)
    d = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
    d[off:off + n].copy_(torch.from_numpy(w.copy()))
    k = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    l = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rc, nt, con, _ = lg.lx_lex_speculative(ctx, ts, trained, d[off:off + n], 0, k, l)
    ek, el, econ = oracle.lex(T.tokenset(NAME), w)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)


def test_speculative_capacity(env, trained):
    # too small an output: LX_E_CAPACITY, the required count, and the first
    # `capacity` tokens written
    import torch
    lg, ctx, ts, S = env
    dfa = T.tokenset(NAME)
    w = corpus.generate(NAME, 20 * 4096, seed=59)
    ek, el, econ = oracle.lex(dfa, w)
    ek, el = oracle.discard(ek, el, T.discarded_kinds(NAME), dfa.n_kinds)
    cap = ek.size // 2
    k = torch.zeros(cap, dtype=torch.int16, device="cuda")
    l = torch.zeros(cap, dtype=torch.int32, device="cuda")
    rc, nt, con, _ = lg.lx_lex_speculative(ctx, ts, trained, _dev(w), 2, k, l)
    assert rc == lg.LX_E_CAPACITY and nt == ek.size and con == econ
    assert np.array_equal(k.cpu().numpy().view(np.uint16).astype(np.int64), ek[:cap])
    assert np.array_equal(l.cpu().numpy().view(np.uint32).astype(np.int64), el[:cap])


def test_full_size_refused_512mib(env, trained):
    """The 512 MiB refused-set workload (C-like with block comments and
    multi-line strings, full stream): the speculative path with the trained
    model and the enumerative path, each compared in full with the oracle."""
    import torch
    lg, ctx, ts, S = env
    w = corpus.generate(NAME)
    n = int(w.size)
    assert n == 512 << 20
    ek, el, econ = oracle.lex(T.tokenset(NAME), w)
    assert econ == n
    d = _dev(w)
    k = torch.zeros(n // 2, dtype=torch.int16, device="cuda")
    l = torch.zeros(n // 2, dtype=torch.int32, device="cuda")
    for path in ("speculative", "enumerative"):
        k.zero_()
        l.zero_()
        if path == "speculative":
            rc, nt, con, st = lg.lx_lex_speculative(ctx, ts, trained, d, 0, k, l)
            assert st["rescanned"] < 0.1 * st["chunks"], st
        else:
            rc, nt, con = lg.lx_lex_enumerative(ctx, ts, d, 0, k, l)
        assert rc == 0 and con == econ and nt == ek.size, (path, rc, con, nt, ek.size)
        assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek), path
        assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el), path


def _adversarial(seed):
    """Block comments and a multi-line string that each span well over 64
    chunks of 4096 bytes, their bodies made of ordinary C-like code (so a
    window inside them looks like code), between stretches of the corpus."""
    base = corpus.generate(NAME, 2 << 20, seed=seed)
    code = corpus.generate("clike", 700_000, seed=seed + 1).tobytes()
    body = code.replace(b"*/", b"* /")
    text = code.replace(b'"', b"'").replace(b"\\", b"/")
    parts = [base[:600_000].tobytes(), b"\n/*", body[:400_000], b"*/\n",
             base[600_000:1_200_000].tobytes(), b'\nx = "', text[:350_000], b'";\n',
             base[1_200_000:].tobytes(), b"\n/*", body[400_000:], b"*/\n"]
    return np.frombuffer(b"".join(parts), np.uint8)


def test_long_cascades_go_to_the_judge(env, trained):
    """Comments and strings spanning hundreds of chunks: the fix-up rounds are
    bounded, the enumerative judge settles the rest, the output is exact."""
    lg, ctx, ts, S = env
    w = _adversarial(71)
    for model in (trained, None):
        for mode in (0, 2):
            st = _check(lg, ctx, ts, model, w, mode)
            assert st["rounds"] <= 9, st
            assert st["judged"], st
    st = _check(lg, ctx, ts, trained, corpus.generate(NAME, 8 << 20, seed=72), 0)
    assert st["rounds"] <= 9, st
