"""CPU reference of the path-gain surrogate MLP (test infrastructure only).

Plain numpy forward and backward of: Fourier features of (tx, rx), ReLU
hidden layers, 2-wide head (path logit, normalised gain), loss = mean of
BCE(logit, has_path) + has_path (gain_norm_pred - gain_norm)^2, and one
Adam step (Kingma & Ba 2015). With bf16=True the values are rounded to
bfloat16 where the GPU stores them in BF16 (features, hidden activations,
weights fed to the GEMMs, back-propagated activation gradients), so the
comparison isolates accumulation order; with bf16=False everything is
float64 (used to pin the backward against finite differences).
Shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

DB_SCALE, DB_OFFSET = 20.0, -100.0


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def unpack(params, F, W, L):
    """Parameter vector -> (weights [L+1], biases [L+1], Fourier matrix)."""
    ws, bs, o = [], [], 0
    for l in range(L + 1):
        fi = 2 * F if l == 0 else W
        fo = 2 if l == L else W
        ws.append(params[o:o + fi * fo].reshape(fo, fi))
        o += fi * fo
        bs.append(params[o:o + fo])
        o += fo
    Bf = params[o:o + 6 * F].reshape(F, 6)
    return ws, bs, Bf


def features(x, Bf, lo, hi, bf16=True):
    xn = 2.0 * (x - lo) / (hi - lo) - 1.0
    a = xn @ Bf.T
    f = np.concatenate([np.sin(2 * np.pi * a), np.cos(2 * np.pi * a)], axis=1)
    return to_bf16(f) if bf16 else f


def forward(params, x, F, W, L, lo, hi, bf16=True):
    dt = np.float32 if bf16 else np.float64
    ws, bs, Bf = unpack(np.asarray(params, dt), F, W, L)
    rnd = to_bf16 if bf16 else (lambda v: v)
    H = [features(np.asarray(x, dt), Bf.astype(dt), lo, hi, bf16).astype(dt)]
    for l in range(L):
        Z = H[-1] @ rnd(ws[l]).T + bs[l]
        H.append(rnd(np.maximum(Z, 0)).astype(dt))
    y = H[-1] @ ws[L].T + bs[L]
    return y, H, ws, bs


def friis_db(x, lam):
    """Free-space gain 20 log10(lam / (4 pi d)) of queries x [n, 6], d = |rx - tx|
    clamped to at least 1 m (the surrogate's optional baseline); 0 if lam == 0."""
    if lam <= 0:
        return np.zeros(len(x))
    d = np.maximum(np.linalg.norm(np.asarray(x, np.float64)[:, 3:] - np.asarray(x, np.float64)[:, :3], axis=1), 1.0)
    return 20.0 * np.log10(lam / (4.0 * np.pi * d))


def gain_db(y, x, lam=0.0):
    """Gain output in dB from the head's second value."""
    return y[:, 1] * DB_SCALE + DB_OFFSET + friis_db(x, lam)


def loss_and_grads(params, x, target, F, W, L, lo, hi, bf16=True, lam=0.0):
    """Mean loss and its gradient (parameter layout; Fourier part zero). With
    lam > 0 the gain head is the residual over the free-space gain."""
    dt = np.float32 if bf16 else np.float64
    rnd = to_bf16 if bf16 else (lambda v: v)
    y, H, ws, bs = forward(params, x, F, W, L, lo, hi, bf16)
    n = len(x)
    z, has = y[:, 0], target[:, 0].astype(dt)
    t = ((target[:, 1].astype(np.float64) - DB_OFFSET - friis_db(x, lam)) / DB_SCALE).astype(dt)
    p = 1.0 / (1.0 + np.exp(-z))
    e = y[:, 1] - t
    loss = np.mean(np.maximum(z, 0) - z * has + np.log1p(np.exp(-np.abs(z))) + has * e * e)
    dy = np.stack([(p - has) / n, 2 * has * e / n], 1).astype(dt)
    gws = [None] * (L + 1)
    gbs = [None] * (L + 1)
    gws[L] = dy.T @ H[L]
    gbs[L] = dy.sum(0)
    dZ = rnd((dy @ ws[L]) * (H[L] > 0))
    for l in range(L - 1, -1, -1):
        gws[l] = dZ.T @ H[l]
        gbs[l] = dZ.sum(0)
        if l > 0:
            dH = dZ @ rnd(ws[l])
            dZ = rnd(dH * (H[l] > 0))
    g = np.concatenate([np.concatenate([gws[l].ravel(), gbs[l].ravel()]) for l in range(L + 1)] +
                       [np.zeros(6 * F, dt)])
    return float(loss), g


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
