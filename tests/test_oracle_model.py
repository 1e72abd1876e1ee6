"""Pins of the FP64 reference of the entry-context model (no GPU): the
analytic gradient against central finite differences on sampled
coordinates of every parameter block, and closed forms (zero hidden layer:
the loss is logsumexp(b2) - b2[y] and its b2 gradient softmax(b2) - onehot)."""

import numpy as np

from oracle import model as M

H, C = 6, 5


def _setup(seed=0, B=7):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, M.n_params(H, C))
    win = rng.integers(0, 257, size=(B, M.W))
    y = rng.integers(0, C, size=B)
    return p, win, y


def test_gradient_matches_finite_differences():
    p, win, y = _setup()
    loss, g = M.loss_and_grad(p, win, y, H, C)
    assert abs(loss - M.loss_only(p, win, y, H, C)) < 1e-12
    rng = np.random.default_rng(1)
    # coordinates from every block: emb rows actually used, W1, b1, W2, b2
    blocks = np.cumsum([0, M.ROWS * M.D, M.W * M.D * H, H, H * C, C])
    used_rows = np.unique(win)
    picks = [int(r) * M.D + d for r in used_rows[:4] for d in (0, 3)]
    for lo, hi in zip(blocks[1:-1], blocks[2:]):
        picks += rng.integers(lo, hi, size=6).tolist()
    eps = 1e-6
    for i in picks:
        q = p.copy(); q[i] += eps
        lp = M.loss_only(q, win, y, H, C)
        q[i] -= 2 * eps
        lm = M.loss_only(q, win, y, H, C)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    # unused embedding rows get no gradient
    unused = np.setdiff1d(np.arange(M.ROWS), used_rows)
    emb_g = g[:M.ROWS * M.D].reshape(M.ROWS, M.D)
    assert np.all(emb_g[unused] == 0)


def test_zero_hidden_layer_closed_form():
    p, win, y = _setup(2)
    emb, W1, b1, W2, b2 = M.split(p, H, C)
    q = p.copy()
    e, w1, bb1, w2, bb2 = M.split(q, H, C)   # views into q
    w1[:] = 0.0
    bb1[:] = -1.0          # every hidden unit off: z = b2 for every window
    loss, g = M.loss_and_grad(q, win, y, H, C)
    sm = np.exp(bb2 - bb2.max()); sm /= sm.sum()
    want = float(np.mean(np.log(np.exp(bb2).sum()) - bb2[y]))
    assert abs(loss - want) < 1e-12
    onehot_mean = np.bincount(y, minlength=C) / len(y)
    gb2 = g[-C:]
    assert np.allclose(gb2, sm - onehot_mean, atol=1e-12)
    # nothing flows below a dead hidden layer
    assert np.all(g[:M.ROWS * M.D + M.W * M.D * H + H] == 0)


def test_windows_padding():
    data = np.arange(10, dtype=np.uint8)
    w = M.windows(data, [0, 5, 9])
    assert w.shape == (3, 64)
    assert w[0, 31] == 256 and w[0, 32] == 0 and w[0, 41] == 9 and w[0, 42] == 256
    assert w[1, 27] == 0 and w[1, 32] == 5
    assert w[2, 23] == 0 and w[2, 32] == 9 and w[2, 33] == 256
