"""Pins of the FP64 reference of the entry-context model (no GPU): the
analytic gradient against central finite differences on sampled
coordinates of every parameter block; closed forms (a dead hidden layer:
the loss is logsumexp(b2) - b2[y] and its b2 gradient softmax(b2) - onehot,
nothing flows below it); the convolution and pooling against a direct
loop over their definitions; the bfloat16 rounding against hand-worked
values."""

import numpy as np

from oracle import model as M

H, C = 6, 5


def _setup(seed=0, B=7):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, M.n_params(H, C))
    win = rng.integers(0, 257, size=(B, M.W))
    y = rng.integers(0, C, size=B)
    return p, win, y


def test_parameter_count_of_the_refused_set_model():
    # F = 32 filters of width 5 over 8-wide embeddings, 64 hidden, 211 contexts
    assert M.n_params(64, 211) == 257 * 8 + 32 * 5 * 8 + 32 + 512 * 64 + 64 + 64 * 211 + 211 == 49915


def test_gradient_matches_finite_differences():
    p, win, y = _setup()
    loss, g = M.loss_and_grad(p, win, y, H, C)
    assert abs(loss - M.loss_only(p, win, y, H, C)) < 1e-12
    rng = np.random.default_rng(1)
    blocks = np.cumsum([0] + M.sizes(H, C))
    used_rows = np.unique(win)
    picks = [int(r) * M.D + d for r in used_rows[:4] for d in (0, 3)]
    for lo, hi in zip(blocks[1:-1], blocks[2:]):
        picks += rng.integers(lo, hi, size=8).tolist()
    eps = 1e-6
    for i in picks:
        q = p.copy(); q[i] += eps
        lp = M.loss_only(q, win, y, H, C)
        q[i] -= 2 * eps
        lm = M.loss_only(q, win, y, H, C)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    unused = np.setdiff1d(np.arange(M.ROWS), used_rows)
    emb_g = g[:M.ROWS * M.D].reshape(M.ROWS, M.D)
    assert np.all(emb_g[unused] == 0)


def test_dead_hidden_layer_closed_form():
    p, win, y = _setup(2)
    q = p.copy()
    emb, Wc, bc, W1, b1, W2, b2 = M.split(q, H, C)   # views into q
    W1[:] = 0.0
    b1[:] = -1.0          # every hidden unit off: z = b2 for every window
    loss, g = M.loss_and_grad(q, win, y, H, C)
    sm = np.exp(b2 - b2.max()); sm /= sm.sum()
    want = float(np.mean(np.log(np.exp(b2).sum()) - b2[y]))
    assert abs(loss - want) < 1e-12
    onehot_mean = np.bincount(y, minlength=C) / len(y)
    assert np.allclose(g[-C:], sm - onehot_mean, atol=1e-12)
    below = sum(M.sizes(H, C)[:5])
    assert np.all(g[:below] == 0)


def test_conv_and_pool_against_direct_loops():
    p, win, y = _setup(3, B=3)
    emb, Wc, bc, W1, b1, W2, b2 = M.split(p, H, C)
    z, (x, h0, hp, a, arg, mf, a1, h1) = M.forward(p, win, H, C)
    for b in range(3):
        for t in (0, 1, 17, 62, 63):
            for f in (0, 5, 31):
                s = bc[f]
                for k in range(M.K):
                    tt = t + k - 2
                    if 0 <= tt < M.W:
                        s += float(np.dot(Wc[f, k], emb[win[b, tt]]))
                assert abs(a[b, t, f] - s) < 1e-12
        for u in (0, 7, 15):
            for f in (2, 30):
                vals = [max(a[b, 4 * u + j, f], 0.0) for j in range(4)]
                assert mf[b, u * M.F + f] == max(vals)
                assert arg[b, u, f] == vals.index(max(vals))   # the first maximum


def test_bf16_rounding_hand_values():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-40])
    got = M.to_bf16(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3 * 2^-8 rounds up to 1 + 2^-6
    assert got.tolist()[:6] == [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0]


def test_windows_padding():
    data = np.arange(10, dtype=np.uint8)
    w = M.windows(data, [0, 5, 9])
    assert w.shape == (3, 64)
    assert w[0, 31] == 256 and w[0, 32] == 0 and w[0, 41] == 9 and w[0, 42] == 256
    assert w[1, 27] == 0 and w[1, 32] == 5
    assert w[2, 23] == 0 and w[2, 32] == 9 and w[2, 33] == 256
