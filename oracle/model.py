"""FP64 reference of the entry-context model -- TEST INFRASTRUCTURE ONLY.

The model scores the context of the serial scan at a chunk start from the 64
bytes around it (the speculative path's predictor; it is not part of the
paper, which only splits at certified bytes): a byte embedding, a 1D
convolution with ReLU, max pooling, and a two-layer MLP.

    h0[t]  = emb[x_t]                      x: 64 byte values, 256 = outside the input
    a[t,f] = bc[f] + sum_{k,d} Wc[f,k,d] h0[t+k-2,d]     (h0 = 0 outside 0..63)
    r      = max(a, 0)
    m[u,f] = max_{t = 4u .. 4u+3} r[t,f]   (the first maximum takes the gradient)
    a1     = m W1 + b1,  h1 = max(a1, 0)   (m flattened as u * F + f)
    z      = h1 W2 + b2
    loss   = mean_b ( logsumexp(z_b) - z_b[y_b] )

Parameters are one flat array in the order emb [257][8], Wc [F][K][8],
bc [F], W1 [16 F][H], b1 [H], W2 [H][C], b2 [C]; with F = 32, K = 5, H = 64
and the 211 contexts of the refused C-like set that is 49 915 parameters.
``loss_and_grad`` is the analytic backward pass; the tests pin it against
central finite differences and against closed forms.
"""

from __future__ import annotations

import numpy as np

W, D, ROWS = 64, 8, 257      # window bytes, embedding width, byte values + pad
F, K, POOL = 32, 5, 4        # filters, kernel width, pool width
U = W // POOL                # pooled positions
PAD = K // 2


def sizes(H: int, C: int):
    return [ROWS * D, F * K * D, F, U * F * H, H, H * C, C]


def split(params: np.ndarray, H: int, C: int):
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    shapes = [(ROWS, D), (F, K, D), (F,), (U * F, H), (H,), (H, C), (C,)]
    for shp in shapes:
        n = int(np.prod(shp))
        out.append(p[o:o + n].reshape(shp))
        o += n
    assert o == p.size
    return out


def n_params(H: int, C: int) -> int:
    return int(sum(sizes(H, C)))


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


def _conv(h0, Wc, bc):
    """a[b, t, f] for the zero-padded sequence h0[b, t, d]."""
    B = h0.shape[0]
    hp = np.zeros((B, W + 2 * PAD, D))
    hp[:, PAD:PAD + W] = h0
    a = np.broadcast_to(bc, (B, W, F)).copy()
    for k in range(K):
        a += np.einsum("btd,fd->btf", hp[:, k:k + W], Wc[:, k, :])
    return a, hp


def forward(params, win, H: int, C: int):
    emb, Wc, bc, W1, b1, W2, b2 = split(params, H, C)
    x = np.asarray(win, dtype=np.int64)
    B = x.shape[0]
    h0 = emb[x]                                   # B, W, D
    a, hp = _conv(h0, Wc, bc)
    r = np.maximum(a, 0.0)
    rp = r.reshape(B, U, POOL, F)
    arg = rp.argmax(axis=2)                       # first maximum
    m = np.take_along_axis(rp, arg[:, :, None, :], axis=2)[:, :, 0, :]   # B, U, F
    mf = m.reshape(B, U * F)
    a1 = mf @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    z = h1 @ W2 + b2
    return z, (x, h0, hp, a, arg, mf, a1, h1)


def loss_and_grad(params, win, labels, H: int, C: int):
    emb, Wc, bc, W1, b1, W2, b2 = split(params, H, C)
    z, (x, h0, hp, a, arg, mf, a1, h1) = forward(params, win, H, C)
    y = np.asarray(labels, dtype=np.int64)
    B = z.shape[0]
    mx = z.max(axis=1, keepdims=True)
    lse = (mx + np.log(np.exp(z - mx).sum(axis=1, keepdims=True)))[:, 0]
    loss = float(np.mean(lse - z[np.arange(B), y]))
    dz = np.exp(z - lse[:, None])
    dz[np.arange(B), y] -= 1.0
    dz /= B
    gW2 = h1.T @ dz
    gb2 = dz.sum(axis=0)
    da1 = (dz @ W2.T) * (a1 > 0)
    gW1 = mf.T @ da1
    gb1 = da1.sum(axis=0)
    dm = (da1 @ W1.T).reshape(B, U, F)
    # pooling: the gradient goes to the first maximum of each window of 4
    dr = np.zeros((B, U, POOL, F))
    np.put_along_axis(dr, arg[:, :, None, :], dm[:, :, None, :], axis=2)
    da = dr.reshape(B, W, F) * (a > 0)
    gbc = da.sum(axis=(0, 1))
    gWc = np.zeros_like(Wc)
    dhp = np.zeros_like(hp)
    for k in range(K):
        gWc[:, k, :] = np.einsum("btf,btd->fd", da, hp[:, k:k + W])
        dhp[:, k:k + W] += np.einsum("btf,fd->btd", da, Wc[:, k, :])
    dh0 = dhp[:, PAD:PAD + W]
    gemb = np.zeros_like(emb)
    np.add.at(gemb, x, dh0)
    grad = np.concatenate([gemb.ravel(), gWc.ravel(), gbc, gW1.ravel(), gb1, gW2.ravel(), gb2])
    return loss, grad


def loss_only(params, win, labels, H: int, C: int) -> float:
    z, _ = forward(params, win, H, C)
    y = np.asarray(labels, dtype=np.int64)
    m = z.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(z - m).sum(axis=1, keepdims=True)))[:, 0]
    return float(np.mean(lse - z[np.arange(z.shape[0]), y]))


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), kept in float64: the
    weights the device computes with."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
