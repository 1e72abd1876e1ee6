"""Failure detection without a GPU fault: a tile that never publishes its
look-back aggregate makes its successors' bounded waits run out; the call
reports LX_E_TIMEOUT within the time budget and the same context then lexes
correctly."""

import time

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


def test_withheld_aggregate_times_out_then_context_recovers(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    ctx = lg.lx_ctx_create()
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    w = corpus.generate("json", 4 << 20, seed=71)
    d = torch.from_numpy(w.copy()).cuda()
    k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
    l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
    assert lg.lx_ctx_set_timeout_ms(ctx, 300) == 0
    assert lg.lx_ctx_debug_withhold(ctx, 5) == 0
    t0 = time.perf_counter()
    rc, _, _ = lg.lx_lex(ctx, ts, d, 2, k, l)
    dt = time.perf_counter() - t0
    assert rc == lg.LX_E_TIMEOUT
    assert dt < 10.0, dt
    # the context is usable again
    assert lg.lx_ctx_debug_withhold(ctx, 0xFFFFFFFF) == 0
    rc, nt, con = lg.lx_lex(ctx, ts, d, 2, k, l)
    ek, el, econ = oracle.lex(T.tokenset("json"), w)
    ek, el = oracle.discard(ek, el, T.discarded_kinds("json"), T.tokenset("json").n_kinds)
    assert rc == 0 and con == econ and nt == ek.size
    assert np.array_equal(k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), ek)
    assert np.array_equal(l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), el)
