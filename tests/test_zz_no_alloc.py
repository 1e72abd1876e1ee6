"""lx_lex_noalloc -- the entry point for callers that cannot allocate.

A caller with a fixed device-memory budget, or one that must not risk the
device synchronization a cudaMalloc can cause while lexing, calls
lx_lex_noalloc instead of lx_lex.  It needs no context and works out of one
fixed device scratch array that every call shares.  Here two such calls in a
row (a larger input, then a smaller malformed one, so stale scratch from the
first call would show) must each reproduce lx_lex's output exactly, the
device's free memory must not move across them, an output buffer that is too
small must give LX_E_CAPACITY with the required count, and an input beyond
the stated maximum is refused before any GPU work.

The cases cover both walk-table forms (JSON: byte-indexed rows; C-like:
class-indexed rows) and a full-stream mode.
"""

import numpy as np
import pytest

from lexinputs import corpus
from lexinputs import tokensets as T

pytestmark = pytest.mark.gpu

CASES = [
    ("json", "FILTERED_MODULO", 0x01),      # 0x01 is invalid in every JSON token
    ("clike", "FILTERED_MODULO", 0x01),     # and outside every C-like token
    ("arith", "FULL_EXACT", ord("?")),      # '?' starts no arith token
]


@pytest.mark.parametrize("name,mode_name,bad", CASES)
def test_noalloc_two_calls_match_lx_lex(lexlib, name, mode_name, bad):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = lexlib
    mode = getattr(lg, "LX_" + mode_name)
    ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    ctx = lg.lx_ctx_create()
    first = corpus.generate(name, 3 << 20, seed=31)
    second = corpus.generate(name, 1 << 20, seed=32).copy()
    second[777777] = bad                            # a lexing error

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

    outs = [(torch.full((d.numel(),), -1, dtype=torch.int16, device="cuda"),
             torch.full((d.numel(),), -1, dtype=torch.int32, device="cuda")) for d in inputs]
    # one warm-up call loads the module and looks up the array's address
    rc, _, _ = lg.lx_lex_noalloc(ts, inputs[1], mode, *outs[1])
    assert rc == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]

    # two allocation-free calls in a row
    results = [lg.lx_lex_noalloc(ts, d, mode, k, l) for d, (k, l) in zip(inputs, outs)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0    # the driver saw no allocation
    for (rc, nt2, con2), (k, l), (nt, con, rk, rl) in zip(results, outs, refs):
        assert rc == 0 and nt2 == nt and con2 == con
        assert np.array_equal(k[:nt].cpu().numpy(), rk)
        assert np.array_equal(l[:nt].cpu().numpy(), rl)

    # too small an output: LX_E_CAPACITY and the count a second call needs
    nt = refs[0][0]
    rc, nt2, con2 = lg.lx_lex_noalloc(ts, inputs[0], mode, *outs[0], capacity=nt // 2)
    assert rc == lg.LX_E_CAPACITY and nt2 == nt and con2 == refs[0][1]

    # beyond the fixed scratch: refused before touching the GPU
    d = inputs[1]
    k = torch.zeros(16, dtype=torch.int16, device="cuda")
    l = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc, _, _ = lg.lx_lex_noalloc(ts, d, mode, k, l, n=lg.LX_NOALLOC_MAX_INPUT + 1)
    assert rc == lg.LX_E_INVAL
