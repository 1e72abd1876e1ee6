"""FP64 reference of the entry-context model -- TEST INFRASTRUCTURE ONLY.

The model scores the context of the serial scan at a chunk start from the 64
bytes around it (the speculative path's predictor; it is not part of the
paper, which only splits at certified bytes):

    h0 = concat_k emb[x_k]            x: 64 byte values, 256 = outside the input
    a1 = h0 W1 + b1,  h1 = max(a1, 0)
    z  = h1 W2 + b2
    loss = mean_b ( logsumexp(z_b) - z_b[y_b] )

Parameters are one flat array in the order emb [257][8], W1 [512][H], b1 [H],
W2 [H][C], b2 [C].  ``loss_and_grad`` is the analytic backward pass; the
tests pin it against central finite differences and against closed forms.
"""

from __future__ import annotations

import numpy as np

W, D, ROWS = 64, 8, 257


def split(params: np.ndarray, H: int, C: int):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    emb = p[o:o + ROWS * D].reshape(ROWS, D); o += ROWS * D
    W1 = p[o:o + W * D * H].reshape(W * D, H); o += W * D * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * C].reshape(H, C); o += H * C
    b2 = p[o:o + C]; o += C
    assert o == p.size
    return emb, W1, b1, W2, b2


def n_params(H: int, C: int) -> int:
    return ROWS * D + W * D * H + H + H * C + C


def windows(data: np.ndarray, positions) -> np.ndarray:
    """64 byte values around each position p: data[p-32 .. p+32), 256 outside."""
    w = np.asarray(data, dtype=np.int64)
    out = np.full((len(positions), W), 256, dtype=np.int64)
    for i, p in enumerate(positions):
        for k in range(W):
            q = int(p) - W // 2 + k
            if 0 <= q < w.size:
                out[i, k] = w[q]
    return out


def forward(params, win, H: int, C: int):
    emb, W1, b1, W2, b2 = split(params, H, C)
    x = np.asarray(win, dtype=np.int64)
    h0 = emb[x].reshape(x.shape[0], W * D)
    a1 = h0 @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    z = h1 @ W2 + b2
    return z, (x, h0, a1, h1)


def loss_and_grad(params, win, labels, H: int, C: int):
    emb, W1, b1, W2, b2 = split(params, H, C)
    z, (x, h0, a1, h1) = forward(params, win, H, C)
    y = np.asarray(labels, dtype=np.int64)
    B = z.shape[0]
    m = z.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(z - m).sum(axis=1, keepdims=True)))[:, 0]
    loss = float(np.mean(lse - z[np.arange(B), y]))
    pr = np.exp(z - lse[:, None])
    dz = pr.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    gW2 = h1.T @ dz
    gb2 = dz.sum(axis=0)
    dh1 = dz @ W2.T
    da1 = dh1 * (a1 > 0)
    gW1 = h0.T @ da1
    gb1 = da1.sum(axis=0)
    dh0 = (da1 @ W1.T).reshape(B, W, D)
    gemb = np.zeros_like(emb)
    np.add.at(gemb, x, dh0)
    grad = np.concatenate([gemb.ravel(), gW1.ravel(), gb1, gW2.ravel(), gb2])
    return loss, grad


def loss_only(params, win, labels, H: int, C: int) -> float:
    z, _ = forward(params, win, H, C)
    y = np.asarray(labels, dtype=np.int64)
    m = z.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(z - m).sum(axis=1, keepdims=True)))[:, 0]
    return float(np.mean(lse - z[np.arange(z.shape[0]), y]))
