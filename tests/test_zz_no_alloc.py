"""lx_lex_noalloc -- the entry point for callers that cannot allocate.

A caller with a fixed device-memory budget, or one that must not risk the
device synchronization a cudaMalloc can cause while lexing, calls
lx_lex_noalloc instead of lx_lex.  It needs no context and works out of one
fixed device scratch array that every call shares.  Here two such calls in a
row (a larger input, then a smaller malformed one, so stale scratch from the
first call would show) must each reproduce lx_lex's output exactly, and an
input beyond the stated maximum is refused before any GPU work.
"""

import numpy as np
import pytest

from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu


def test_noalloc_two_calls_match_lx_lex(lexlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    mode = lg.LX_FILTERED_MODULO
    ts = lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json"))
    ctx = lg.lx_ctx_create()
    first = corpus.generate("json", 3 << 20, seed=31)
    second = corpus.generate("json", 1 << 20, seed=32).copy()
    second[777777] = 0x01                           # invalid in every JSON token: a lexing error

    inputs, refs = [], []
    for w in (first, second):
        d = torch.from_numpy(w.copy()).cuda()
        k = torch.zeros(w.size, dtype=torch.int16, device="cuda")
        l = torch.zeros(w.size, dtype=torch.int32, device="cuda")
        rc, nt, con = lg.lx_lex(ctx, ts, d, mode, k, l)
        assert rc == 0
        inputs.append(d)
        refs.append((nt, con, k[:nt].cpu().numpy(), l[:nt].cpu().numpy()))
    assert refs[1][1] <= 777777

    # two allocation-free calls in a row
    outs = []
    for d in inputs:
        k = torch.full((d.numel(),), -1, dtype=torch.int16, device="cuda")
        l = torch.full((d.numel(),), -1, dtype=torch.int32, device="cuda")
        outs.append((lg.lx_lex_noalloc(ts, d, mode, k, l), k, l))
    for (rc_nt_con, k, l), (nt, con, rk, rl) in zip(outs, refs):
        rc, nt2, con2 = rc_nt_con
        assert rc == 0 and nt2 == nt and con2 == con
        assert np.array_equal(k[:nt].cpu().numpy(), rk)
        assert np.array_equal(l[:nt].cpu().numpy(), rl)

    # beyond the fixed scratch: refused before touching the GPU
    d = inputs[1]
    k = torch.zeros(16, dtype=torch.int16, device="cuda")
    l = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc, _, _ = lg.lx_lex_noalloc(ts, d, mode, k, l, n=lg.LX_NOALLOC_MAX_INPUT + 1)
    assert rc == lg.LX_E_INVAL
