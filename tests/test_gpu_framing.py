"""A framed refused-set document (0x1E before every line or comment, Section
7.1) lexed by lx_lex on the certified path, against the oracle: the full
stream against the serial scan of the framed document, and the kept stream
(whitespace, comments and frames discarded) against the serial scan of the
same document with its frames deleted."""

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


def test_framed_document(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    dfa = T.tokenset("clike_block")
    I = T.discarded_kinds("clike_block")
    ts_full = lg.lx_compile_tokenset_framed(dfa, I, T.FRAME)
    ts_kept = lg.lx_compile_tokenset_framed(dfa, I, T.FRAME, frame_discarded=True)
    ctx = lg.lx_ctx_create()
    w = corpus.generate("clike_block_framed", 16 << 20, seed=11)
    d = torch.from_numpy(w.copy()).cuda()
    k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size, dtype=torch.int32, device="cuda")

    rc, nt, con = lg.lx_lex(ctx, ts_full, d, lg.LX_FULL_EXACT, k, l)
    ek, el, econ = oracle.lex(T.framed(dfa), w)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)

    u = w[w != T.FRAME]
    uk, ul, ucon = oracle.lex(dfa, u)
    uk, ul = oracle.discard(uk, ul, I, dfa.n_kinds)
    for mode in (lg.LX_FILTERED_EXACT, lg.LX_FILTERED_MODULO):
        rc, nt, con = lg.lx_lex(ctx, ts_kept, d, mode, k, l)
        assert rc == 0 and con == w.size and nt == uk.size
        assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), uk)
        assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), ul)
