"""CPU oracle of the learned proposal net (not part of the paper's method).

TEST INFRASTRUCTURE ONLY: used by the tests to check the GPU net kernels; the
library never imports it. Plain numpy in float64, written from the definitions:
3x3 convolutions with dilation and zero padding, ReLU, the relaxed
winner-takes-all L1 loss, their gradients by the chain rule, and Adam
(Kingma & Ba, 2015). BF16 rounding is applied at the same points as the GPU
kernels (convolution operands), so results match up to FP32 accumulation order.
"""
from __future__ import annotations

import numpy as np

LAYERS = 4


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even) and return float64.

    bfloat16 keeps the upper 16 bits of an IEEE binary32; rounding to nearest
    even adds 0x7FFF plus the lowest kept bit before truncating. Inputs are first
    rounded to binary32 (the GPU converts from float)."""
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def shapes(desc):
    ch = [desc["cin"], desc["c1"], desc["c2"], desc["c3"], 2 * desc["k"]]
    out, off = [], 0
    for l in range(LAYERS):
        cin, cout = ch[l], ch[l + 1]
        out.append(dict(cin=cin, cout=cout, dil=desc["dil"][l], woff=off, boff=off + cout * cin * 9))
        off += cout * cin * 9 + cout
    return out, off


def unpack(params, desc):
    sh, _ = shapes(desc)
    Ws, bs = [], []
    for s in sh:
        Ws.append(np.asarray(params[s["woff"]:s["boff"]], np.float64).reshape(s["cout"], s["cin"], 3, 3))
        bs.append(np.asarray(params[s["boff"]:s["boff"] + s["cout"]], np.float64))
    return Ws, bs


def conv(a, W, b, dil):
    """out[b][n][y][x] = bias[n] + sum_{c,ky,kx} W[n][c][ky][kx] a[b][c][y+(ky-1)d][x+(kx-1)d],
    zero outside the image."""
    B, C, H, Wd = a.shape
    N = W.shape[0]
    d = dil
    ap = np.zeros((B, C, H + 2 * d, Wd + 2 * d))
    ap[:, :, d:d + H, d:d + Wd] = a
    out = np.zeros((B, N, H, Wd)) + (0 if b is None else b[None, :, None, None])
    for ky in range(3):
        for kx in range(3):
            sl = ap[:, :, ky * d:ky * d + H, kx * d:kx * d + Wd]
            out += np.einsum("nc,bcyx->bnyx", W[:, :, ky, kx], sl)
    return out


def conv_input_grad(g, W, dil, H, Wd):
    """Gradient of conv's output w.r.t. its input: the adjoint of conv."""
    B, N, _, _ = g.shape
    C = W.shape[1]
    d = dil
    gp = np.zeros((B, C, H + 2 * d, Wd + 2 * d))
    for ky in range(3):
        for kx in range(3):
            gp[:, :, ky * d:ky * d + H, kx * d:kx * d + Wd] += np.einsum("nc,bnyx->bcyx", W[:, :, ky, kx], g)
    return gp[:, :, d:d + H, d:d + Wd]


def conv_weight_grad(g, a, dil):
    B, C, H, Wd = a.shape
    N = g.shape[1]
    d = dil
    ap = np.zeros((B, C, H + 2 * d, Wd + 2 * d))
    ap[:, :, d:d + H, d:d + Wd] = a
    dW = np.zeros((N, C, 3, 3))
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("bnyx,bcyx->nc", g, ap[:, :, ky * d:ky * d + H, kx * d:kx * d + Wd])
    return dW, g.sum(axis=(0, 2, 3))


def forward(params, x, desc, rounding=True):
    """Returns out and the per-layer (input activation, pre-activation) list."""
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    sh, _ = shapes(desc)
    Ws, bs = unpack(params, desc)
    a = rnd(x)
    cache = []
    for l, s in enumerate(sh):
        pre = conv(a, rnd(Ws[l]), bs[l], s["dil"])
        cache.append((a, pre))
        if l < LAYERS - 1:
            a = rnd(np.maximum(pre, 0))
    return pre, cache


def backward(params, dout, cache, desc, rounding=True):
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    sh, n = shapes(desc)
    Ws, _ = unpack(params, desc)
    grads = np.zeros(n)
    g = rnd(dout)
    for l in range(LAYERS - 1, -1, -1):
        a, pre = cache[l]
        dW, db = conv_weight_grad(g, a, sh[l]["dil"])
        s = sh[l]
        grads[s["woff"]:s["boff"]] = dW.ravel()
        grads[s["boff"]:s["boff"] + s["cout"]] = db
        if l == 0:
            break
        H, Wd = a.shape[2:]
        gin = conv_input_grad(g, rnd(Ws[l]), s["dil"], H, Wd)
        g = rnd(gin * (cache[l - 1][1] > 0))
    return grads


def wta_loss(out, label, valid, K, scale, alpha):
    """Relaxed WTA L1: per labelled point, weight 1-alpha on the candidate nearest
    to the label (L1, first on ties), alpha/(K-1) on the others; mean over
    labelled points. Returns (loss, dloss/dout)."""
    B, _, Gy, Gx = out.shape
    lx = label[..., 0] / scale
    ly = label[..., 1] / scale
    o = out.reshape(B, K, 2, Gy, Gx)
    e = np.abs(o[:, :, 0] - lx[:, None]) + np.abs(o[:, :, 1] - ly[:, None])
    best = np.argmin(e, axis=1)  # first minimum on ties
    w = np.full((B, K, Gy, Gx), alpha / (K - 1) if K > 1 else 1.0)
    np.put_along_axis(w, best[:, None], 1.0 - alpha if K > 1 else 1.0, axis=1)
    v = valid.astype(bool)
    cnt = max(int(v.sum()), 1)
    loss = float((w * e)[np.broadcast_to(v[:, None], e.shape)].sum()) / cnt
    d = np.zeros_like(o)
    d[:, :, 0] = w * np.sign(o[:, :, 0] - lx[:, None])
    d[:, :, 1] = w * np.sign(o[:, :, 1] - ly[:, None])
    d *= v[:, None, None] / cnt
    return loss, d.reshape(out.shape)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def net_input(I1, I2, n=8):
    """Rounded mean of each n x n block per channel, v / 255 - 0.5; [6][Gy][Gx]."""
    out = []
    for img in (I1, I2):
        H, W = img.shape[:2]
        Gy, Gx = -(-H // n), -(-W // n)
        for c in range(3):
            ch = np.zeros((Gy, Gx))
            for j in range(Gy):
                for i in range(Gx):
                    blk = img[j * n:(j + 1) * n, i * n:(i + 1) * n, c].astype(np.int64)
                    s, cnt = int(blk.sum()), blk.size
                    # float32 arithmetic, as the GPU computes it
                    ch[j, i] = np.float32((s + cnt // 2) // cnt) / np.float32(255) - np.float32(0.5)
            out.append(ch)
    return np.stack(out)
