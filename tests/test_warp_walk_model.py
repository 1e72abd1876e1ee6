"""Host model of the warp-tile lexer (lexwarp.cu) over the event-code walk
tables of ``lx_tokenset_walk_table``, checked against the oracle.

The model follows the kernel step for step, with the lanes of a warp run one
after the other (each input position has exactly one owning lane, so the
order does not matter): lanes start their slices in the PRE row, step whole
16-byte blocks, store the packed event codes of words that did not begin in
PRE (and, byte by byte, the codes after the first certified byte of the word
where PRE was left), take the next lane's first certified byte (or the first
one past the tile, found by a scan of the halo) as their range end, store
nothing past it, replay a token from q0 on reaching SLOW (longest match with
backtracking), and finish at the end of the input.  Counting and emission
read the event codes of (c0, hi] in order; a last range that leaves the
halo is walked byte by byte.  The geometry is a parameter, so small tiles
exercise every edge on short inputs.
"""

import random

import numpy as np
import pytest

import oracle
from lexinputs import corpus
from lexinputs import tokensets as T

NONE = 0xFFFFFFFF


class Walk:
    def __init__(self, blob, meta):
        self.blob = blob
        self.form = meta["form"]
        self.shift = meta["row_shift"]
        self.ent = blob[:meta["n_rows"] << self.shift].view(np.uint16).astype(np.int64)
        self.P_start, self.P_pre, self.P_slow = meta["p_start"], meta["p_pre"], 0
        self.acc = blob[meta["acc_off"]:meta["acc_off"] + meta["n_rows"]].astype(np.int64)
        self.kmap = blob[meta["kmap_off"]:meta["kmap_off"] + 256].view(np.uint16).astype(np.int64)
        self.cmap2 = blob[meta["cmap_off"]:meta["cmap_off"] + 256].astype(np.int64)
        self.K = meta.get("n_ctx", 0)
        self.cuts = blob[meta["cut_off"]:meta["cut_off"] + 256 * (self.K + 1)].astype(bool).reshape(self.K + 1, 256)
        self.ctx = (blob[meta["ctx_off"]:meta["ctx_off"] + 256].astype(np.int64) if self.K
                    else np.zeros(256, np.int64))

    def is_cut(self, a, b):
        """A chunk may start at byte b after byte a (single byte or window)."""
        return bool(self.cuts[self.ctx[a], b])

    def is_pre(self, e):
        return e >= self.P_pre          # PRE and the PRE_k rows after it

    def step(self, e, b):
        if self.form == 0:
            a = (e & ~0x1FE) | (b << 1)
        else:
            a = (e & ~0xFF) | int(self.cmap2[b])
        return int(self.ent[a >> 1])

    def acc_code(self, e):
        return int(self.acc[e >> self.shift])


class WarpModel:
    def __init__(self, walk, wt=6144, halo=512, blk=16):
        self.W = walk
        self.WT, self.SLICE, self.HALO, self.BLK = wt, wt // 32, halo, blk
        self.EVB = wt + halo
        self.LIMIT = self.EVB - blk

    # one lane's SLOW handling: replay its token from the token start, then
    # re-walk to `upto`.  Only positions <= hi are stored; a SLOW entered past
    # hi belongs to the next range and just stops the lane.
    def slow_fix(self, L, upto, hi):
        W = self.W
        while True:
            tok = L["s"]
            for j in range(min(upto - 1, hi), L["s"], -1):
                if self.ev[j]:
                    tok = j
                    break
            q, r, rc = W.P_start, None, 0
            for k in range(tok, upto):
                v = W.step(q, self.inb(k))
                if (v & 0xFF) or v == W.P_slow:
                    break
                q = v
                ac = W.acc_code(q)
                if ac:
                    r, rc = k + 1, ac
            if r is None:
                if tok < L["own_hi"]:
                    L["fail"] = tok
                L["act"] = False
                return
            if r <= hi:
                self.ev[r] = rc
            e, kslow = W.P_start, None
            for k in range(r, upto):
                v = W.step(e, self.inb(k))
                if r < k <= hi:          # the step at r (from START) ends nothing
                    self.ev[k] = v & 0xFF
                if v == W.P_slow and e != W.P_slow:
                    kslow = k
                e = v
            L["e"] = e
            if e != W.P_slow:
                return
            if kslow > hi or r > hi:
                L["act"] = False
                return

    def finalize(self, L, hi):
        # at the end of the input: an accepting row ends its token there
        W = self.W
        if self.nrel > hi:
            L["act"] = False
            return
        while L["act"]:
            e = L["e"]
            if e == W.P_start or W.is_pre(e):
                return
            if e != W.P_slow:
                ac = W.acc_code(e)
                if ac:
                    self.ev[self.nrel] = ac
                    return
                L["e"] = W.P_slow
            self.slow_fix(L, self.nrel, hi)

    def scalar(self, L, upto, hi):
        # byte steps up to `upto` with the kernel's storing rule
        W = self.W
        while L["p"] < upto and L["act"]:
            k = L["p"]
            e0 = L["e"]
            v = W.step(e0, self.inb(k))
            if W.is_pre(e0) and not W.is_pre(v) and L["s"] == NONE:
                L["s"] = k
            if not W.is_pre(e0) and k <= hi:
                self.ev[k] = v & 0xFF
            L["e"] = v
            L["p"] = k + 1
            if v == W.P_slow:
                if k > hi:
                    L["act"] = False
                    return
                self.slow_fix(L, k + 1, hi)

    def block(self, L, hi_rule):
        """One lockstep block: 4 words, packed stores.  hi_rule: None (phase 1,
        store words that did not begin in PRE) or the range end (phase 2,
        store whole words at or before it)."""
        W = self.W
        pb = L["p"]
        e_in = L["e"]
        words = []
        for wk in range(self.BLK // 4):
            e0 = L["e"]
            codes = []
            for k in range(4):
                L["e"] = W.step(L["e"], self.inb(pb + 4 * wk + k))
                codes.append(L["e"] & 0xFF)
            words.append((e0, codes))
            wpos = pb + 4 * wk
            if (hi_rule is None and not W.is_pre(e0)) or (hi_rule is not None and wpos + 3 <= hi_rule):
                self.ev[wpos:wpos + 4] = codes
        if hi_rule is None and L["s"] == NONE and not W.is_pre(L["e"]):
            # PRE was left in this block: the byte where the PRE rows are left starts the range
            e, s = e_in, None
            for k in range(pb, pb + self.BLK):
                e = W.step(e, self.inb(k))
                if not W.is_pre(e):
                    s = k
                    break
            L["s"] = s
            wk = (s - pb) // 4
            for j in range(s + 1, pb + 4 * wk + 4):
                self.ev[j] = words[wk][1][j - pb - 4 * wk]
        L["p"] = pb + self.BLK
        return words

    def inb(self, k):
        return int(self.w[self.tb + k])

    def generic(self, start, emit):
        """The last range when it leaves the halo: byte steps from the
        certified byte at `start` to the first certified byte at or past the
        tile end (or the end of the input).  Returns (count, fail)."""
        W = self.W
        e, p, tok, cnt = W.P_start, start, start, 0
        while True:
            if p == self.nrel:
                if e == W.P_start:
                    return cnt, NONE
                ac = W.acc_code(e) if e != W.P_slow else 0
                if ac:
                    cnt += self._emit(emit, ac, p - tok)
                    return cnt, NONE
                slow = True
            else:
                b = self.inb(p)
                v = W.step(e, b)
                slow = v == W.P_slow
                if not slow:
                    if v & 0xFF:
                        cnt += self._emit(emit, v & 0xFF, p - tok)
                        tok = p
                        if p >= self.WT and W.is_cut(self.inb(p - 1), b):
                            return cnt, NONE
                    e = v
                    p += 1
                    continue
            q, r, rc = W.P_start, None, 0
            for k in range(tok, p):
                v = W.step(q, self.inb(k))
                if (v & 0xFF) or v == W.P_slow:
                    break
                q = v
                if W.acc_code(q):
                    r, rc = k + 1, W.acc_code(q)
            if r is None:
                return cnt, tok
            cnt += self._emit(emit, rc, r - tok)
            tok = p = r
            e = W.P_start
            if r == self.nrel:
                return cnt, NONE
            if r >= self.WT and W.is_cut(self.inb(r - 1), self.inb(r)):
                return cnt, NONE

    def _emit(self, emit, code, ln):
        if code >= 4:
            if emit is not None:
                emit.append((int(self.W.kmap[code >> 1]), ln))
            return 1
        return 0

    def tile(self, w, tile):
        W = self.W
        self.w = w
        self.tb = tile * self.WT
        n = int(w.size)
        self.nrel = nrel = n - self.tb
        self.ev = np.zeros(self.EVB + 16, np.int64)
        # c1: the first certified byte at or past the tile end, inside the halo
        if nrel <= self.WT:
            c1 = nrel
        else:
            lim = min(nrel, self.LIMIT)
            c1 = next((k for k in range(self.WT, lim) if W.is_cut(self.inb(k - 1), self.inb(k))), NONE)
            if c1 == NONE and lim == nrel:
                c1 = nrel
        lanes = []
        for l in range(32):
            t0 = l * self.SLICE
            first = tile == 0 and l == 0
            pre0 = W.P_pre
            if W.K and not first and t0 < nrel:
                pre0 += int(W.ctx[self.inb(t0 - 1)]) << W.shift    # the context of the byte before the slice
            L = dict(p=t0, e=W.P_start if first else pre0, s=0 if first else NONE, fail=NONE,
                     act=t0 < nrel, own_hi=NONE)
            lanes.append(L)
        # phase 1
        for l, L in enumerate(lanes):
            end1 = (l + 1) * self.SLICE
            L["own_hi"] = NONE
            while L["act"] and L["p"] < end1:
                if L["p"] + self.BLK <= nrel:
                    self.block(L, None)
                    if L["e"] == W.P_slow:
                        self.slow_fix(L, L["p"], 1 << 40)
                else:
                    self.scalar(L, nrel, 1 << 40)
                    self.finalize(L, 1 << 40)
                    L["act"] = False
        s = [L["s"] for L in lanes]
        ends = []
        for l in range(32):
            nxt = min([x for x in s[l + 1:] if x != NONE], default=NONE)
            ends.append(c1 if nxt == NONE else nxt)
        have = [x for x in s if x != NONE]
        c0 = min(have) if have else NONE
        long_s = NONE
        # phase 2
        for l, L in enumerate(lanes):
            end = ends[l]
            if s[l] == NONE or not L["act"]:
                continue
            if end == NONE:
                long_s = s[l]
                continue
            L["own_hi"] = end
            while L["act"] and L["p"] <= end:
                if L["p"] + self.BLK <= nrel:
                    pb = L["p"]
                    words = self.block(L, end)
                    if L["p"] > end:
                        wk = (end - pb) // 4
                        wpos = pb + 4 * wk
                        for j in range(wpos, end + 1):
                            self.ev[j] = words[wk][1][j - wpos]
                        if L["e"] == W.P_slow and self.ev[end] == 0:
                            self.slow_fix(L, L["p"], end)
                        L["act"] = False
                    elif L["e"] == W.P_slow:
                        self.slow_fix(L, L["p"], end)
                else:
                    self.scalar(L, nrel, end)
                    self.finalize(L, end)
                    L["act"] = False
        fails = [L["fail"] for L in lanes]
        fail = min(fails)
        out = []
        if c0 == NONE:
            return out, NONE, False
        hi = c1 if long_s == NONE else long_s
        if fail < hi:
            hi = fail
        prev = c0
        for p in range(c0 + 1, hi + 1):
            code = int(self.ev[p])
            if code:
                if code >= 4:
                    out.append((int(W.kmap[code >> 1]), p - prev))
                prev = p
        assert self.emit_words(c0, hi) == out
        if long_s != NONE and fail > long_s:
            _, f2 = self.generic(long_s, out)
            fail = f2 if f2 != NONE else fail
        return out, fail, True


    def emit_words(self, c0, hi):
        """The kernel's emission: the words holding positions c0 + 1 .. hi
        split into 32 contiguous lane ranges; each lane starts from the last
        event of the lanes before it (or c0) and runs four bytes per word with
        a 32-bit wrapping distance, of which the stage keeps the low 16 bits."""
        W = self.W
        ev = np.zeros(len(self.ev) + 4, np.int64)
        ev[:len(self.ev)] = self.ev
        ev[hi + 1:] = 0          # the kernel clears the codes after hi when hi is not the halo's byte
        w0, w1 = (c0 + 1) >> 2, max((hi >> 2) + 1, (c0 + 1) >> 2)
        per = (w1 - w0 + 31) // 32
        lanes = [(min(w0 + i * per, w1), min(min(w0 + i * per, w1) + per, w1)) for i in range(32)]
        last = []
        for wa, wb in lanes:
            nz = [p for p in range(4 * wa, 4 * wb) if ev[p]]
            last.append(nz[-1] if nz else 0)
        out = []
        for i, (wa, wb) in enumerate(lanes):
            prev = max(last[:i], default=0)
            if i == 0 or prev < c0:
                prev = c0
            d = (4 * wa - prev) & 0xFFFFFFFF
            for p in range(4 * wa, 4 * wb):
                c = int(ev[p])
                if c > 3:
                    out.append((int(W.kmap[c >> 1]), d & 0xFFFF))
                if c:
                    d = 0
                d = (d + 1) & 0xFFFFFFFF
        return out


def model_lex(lg, name, mode, w, **geo):
    ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    rc, blob, meta = lg.lx_tokenset_walk_table(ts, mode)
    assert rc == 0, rc
    m = WarpModel(Walk(blob, meta), **geo)
    n = int(w.size)
    toks = []
    n_tiles = (n + m.WT - 1) // m.WT
    for t in range(n_tiles):
        out, fail, _ = m.tile(w, t)
        if fail != NONE:
            # the tokens before the failure, and nothing after it (Corollary 1)
            return toks + out, t * m.WT + fail
        toks += out
    return toks, n


def expected(name, mode, w):
    dfa = T.tokenset(name)
    k, l, con = oracle.lex(dfa, w)
    if mode:
        k, l = oracle.discard(k, l, T.discarded_kinds(name), dfa.n_kinds)
    return list(zip(k.tolist(), l.tolist())), con


SMALL = dict(wt=512, halo=128, blk=16)   # 16-byte slices: one block per lane


@pytest.fixture(scope="module")
def lg(lexlib):
    return lexlib


@pytest.mark.parametrize("name,mode", [("arith", 0), ("arith", 2), ("json", 2), ("clike", 2), ("clike_row1", 0),
                                       ("json", 0), ("json", 1), ("clike", 0), ("clike", 1)])
def test_model_matches_oracle_corpora(lg, name, mode):
    gen = "clike" if name == "clike_row1" else name
    w = corpus.generate(gen, 20000, seed=11)
    got, con = model_lex(lg, name, mode, w, **SMALL)
    want, econ = expected(name, mode, w)
    assert con == econ and got == want


@pytest.mark.parametrize("name,mode", [("json", 2), ("clike", 2), ("arith", 0)])
def test_model_full_geometry(lg, name, mode):
    w = corpus.generate(name, 3 * 6144 + 999, seed=12)
    got, con = model_lex(lg, name, mode, w)
    want, econ = expected(name, mode, w)
    assert con == econ and got == want


def test_model_errors_long_lines_and_ragged(lg):
    rng = random.Random(5)
    base = corpus.generate("json", 6000, seed=13)
    for n in (1, 15, 16, 17, 255, 256, 257, 300, 511, 600, 6000):
        w = base[:n]
        got, con = model_lex(lg, "json", 2, w, **SMALL)
        assert (got, con) == expected("json", 2, w), n
    for _ in range(12):
        w = base.copy()
        w[rng.randrange(w.size)] = 0x01
        got, con = model_lex(lg, "json", 2, w, **SMALL)
        assert (got, con) == expected("json", 2, w)
    # lines longer than the halo: the last range leaves it
    line = b'{"k":"' + b"x" * 700 + b'"}\n'
    w = np.frombuffer(line * 6 + base[:900].tobytes(), np.uint8)
    got, con = model_lex(lg, "json", 2, w, **SMALL)
    assert (got, con) == expected("json", 2, w)


def test_model_backtracking(lg):
    # '..' in C-like backtracks from the '...' prefix; '0x' from a hex prefix;
    # arith '===' is '==' then '='
    rng = random.Random(6)
    parts = [b"a..b", b"0x", b"x...y", b"1.", b".5", b"a->b", b"a-->b", b" ", b"\n", b";"]
    w = np.frombuffer(b"".join(rng.choice(parts) for _ in range(3000)), np.uint8)
    got, con = model_lex(lg, "clike", 2, w, **SMALL)
    assert (got, con) == expected("clike", 2, w)
    w = np.frombuffer(b"".join(rng.choice([b"===", b"=", b"==", b"a", b"\n", b"(", b" "]) for _ in range(3000)),
                      np.uint8)
    got, con = model_lex(lg, "arith", 0, w, **SMALL)
    assert (got, con) == expected("arith", 0, w)


def test_walk_table_codes(lg):
    # every event code of a transition is the code of the kind its row accepts
    ts = lg.lx_compile_tokenset(T.tokenset("clike"), T.discarded_kinds("clike"))
    rc, blob, meta = lg.lx_tokenset_walk_table(ts, 2)
    assert rc == 0 and meta["form"] == 1
    W = Walk(blob, meta)
    for r in range(meta["n_rows"]):
        e = r << W.shift
        for b in range(256):
            v = W.step(e, b)
            if v & 0xFF:
                assert W.acc_code(e) == v & 0xFF
    rc, blob, meta = lg.lx_tokenset_walk_table(lg.lx_compile_tokenset(T.tokenset("json"), T.discarded_kinds("json")), 2)
    assert rc == 0 and meta["form"] == 0


@pytest.mark.parametrize("name,mode", [("arith", 0), ("arith", 1), ("json", 2), ("json", 1), ("clike", 2),
                                       ("clike_row1", 0), ("clike_row1", 2), ("json", 0), ("clike", 1)])
def test_model_random_snippets(lg, name, mode):
    """Random slices of the corpora (some with a malformed byte) at every
    alignment, tile and slice boundary of the small geometry."""
    gen = "clike" if name == "clike_row1" else name
    base = corpus.generate(gen, 1 << 16, seed=21)
    rng = random.Random(hash((name, mode)) & 0xFFFF)
    for _ in range(60):
        a = rng.randrange(0, len(base) - 1300)
        s = bytearray(base[a:a + rng.randint(1, 1300)])
        if rng.random() < 0.3 and s:
            s[rng.randrange(len(s))] = rng.choice(b"\x01`@#$\x7f")
        w = np.frombuffer(bytes(s), np.uint8)
        got, con = model_lex(lg, name, mode, w, **SMALL)
        assert (got, con) == expected(name, mode, w), (a, len(s))


@pytest.mark.parametrize("name,mode", [("json", 0), ("json", 1), ("clike", 0), ("arith", 0)])
def test_window_rows(lg, name, mode):
    """In the exact modes the walk table holds PRE_k rows for the split-window
    contexts: PRE_k leaves the PRE rows exactly on the bytes its cut-table row
    certifies (as q0's step), and otherwise moves to the PRE row of the byte's
    own context."""
    ts = lg.lx_compile_tokenset(T.tokenset(name), T.discarded_kinds(name))
    rc, blob, meta = lg.lx_tokenset_walk_table(ts, mode)
    assert rc == 0
    W = Walk(blob, meta)
    rc, pairs = lg.lx_window_certificates(ts)
    if name in ("json", "clike"):
        assert W.K > 0
    for k in range(W.K + 1):
        row = W.P_pre + (k << W.shift)
        for b in range(256):
            v = W.step(row, b)
            if W.cuts[k, b]:
                assert v == W.step(W.P_start, b)
            else:
                assert v == W.P_pre + (int(W.ctx[b]) << W.shift)
    # every context's row certifies exactly the window followers of its bytes (plus single cuts)
    single = W.cuts[0]
    for a in range(256):
        k = int(W.ctx[a])
        if k:
            assert np.array_equal(W.cuts[k], pairs[a] | single)


@pytest.mark.parametrize("name,mode", [("json", 2), ("clike", 0)])
def test_model_dense_geometry(lg, name, mode):
    # the dense geometry's 2048-position halo: lines of 600-1500 bytes leave
    # the sparse halo but end inside this one
    rng = random.Random(14)
    base = corpus.generate(name, 3 * 6144, seed=15).tobytes()
    filler = b'"' + b"q" * 20 + b'"' if name == "json" else b"x" * 20
    long_lines = b"".join((b"[" + filler * rng.randint(30, 70) + b"]\n") if name == "json"
                          else (filler * rng.randint(30, 70) + b";\n") for _ in range(12))
    w = np.frombuffer(base[:7000] + long_lines + base[7000:], np.uint8)
    got, con = model_lex(lg, name, mode, w, wt=6144, halo=2048)
    want, econ = expected(name, mode, w)
    assert con == econ and got == want


def stage_split(counts, cap):
    """The dense emission's placement: lanes whose codes all fit the stage
    (a prefix, since the inclusive counts ascend) write it from their
    exclusive prefix, the others the spill slot from the first misfit lane's
    prefix on.  Returns (split, [(lane, 'stage'|'spill', first index)])."""
    excl = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(int)
    fit = int(np.sum(excl + np.asarray(counts) <= cap))
    total = int(np.sum(counts))
    split = total if fit == len(counts) else int(excl[fit])
    return split, [(i, "stage" if i < fit else "spill", int(excl[i]) if i < fit else int(excl[i]) - split)
                   for i in range(len(counts))]


def test_stage_split_and_copy_groups():
    rng = random.Random(16)
    for _ in range(400):
        cap = rng.choice([768, 1536])
        counts = [rng.choice([0, rng.randint(0, 30), rng.randint(0, 200)]) for _ in range(32)]
        total = sum(counts)
        split, place = stage_split(counts, cap)
        assert split <= cap and split <= total
        stage, spill = {}, {}
        for (lane, where, first), c in zip(place, counts):
            for k in range(c):
                (stage if where == "stage" else spill)[first + k] = (lane, k)
        assert max(stage, default=-1) < cap and len(stage) == split and len(spill) == total - split
        # the copy reads stage[0:split] then spill[0:total-split]: every token once, in lane order
        order = [stage[i] for i in range(split)] + [spill[i] for i in range(total - split)]
        assert order == [(lane, k) for lane in range(32) for k in range(counts[lane])]
    # copy groups: the lanes' groups of V, the tokens before and after them, cover [0, staged) once
    for V in (2, 4):
        for G in range(0, 9):
            for staged in range(0, 200):
                h = min((V - (G & (V - 1))) & (V - 1), staged)
                ng = (staged - h) // V
                t = h + V * ng
                cover = list(range(h)) + [h + V * q + j for q in range(ng) for j in range(V)] + list(range(t, staged))
                assert sorted(cover) == list(range(staged)) and staged - t < V
                assert all((G + h + V * q) % V == 0 for q in range(ng))
