"""FP64 reference of the retention-count predictor -- TEST INFRASTRUCTURE ONLY.

Plain numpy forward and backward pass of the network the library trains
(4 convolutions of width 5 with zero "same" padding and zero beyond each
sequence's length, 32 -> 128 -> 128 -> 128 -> 8 channels, ReLU after the
first three, mean squared error over the valid (position, band) entries),
written from that definition with explicit per-tap matrix products.  With
``bf16=True`` the weights and every layer input are rounded to bfloat16
(round to nearest, ties to even) as the device kernels store them, so device
gradients can be compared with it; with ``bf16=False`` it is pure FP64 and its
gradient is pinned by finite differences in the tests.

Parameter layout (flat, as sd_pred_get_params returns it): for each layer,
W[5][cin][cout] then bias[cout].
"""
from __future__ import annotations

import numpy as np

CIN = (32, 128, 128, 128)
COUT = (128, 128, 128, 8)
TAPS = 5


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params: np.ndarray):
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for cin, cout in zip(CIN, COUT):
        w = p[off:off + TAPS * cin * cout].reshape(TAPS, cin, cout)
        off += TAPS * cin * cout
        b = p[off:off + cout]
        off += cout
        out.append((w, b))
    assert off == p.size
    return out


def _mask(B, L, lengths):
    pos = np.arange(L)[None, :]
    return (pos < np.asarray(lengths)[:, None]).astype(np.float64)  # (B, L)


def _conv(x, w):
    """z[b,l,co] = sum_t sum_ci x[b, l+t-2, ci] w[t, ci, co] (zero outside)."""
    B, L, _ = x.shape
    z = np.zeros((B, L, w.shape[2]))
    for t in range(TAPS):
        s = t - 2
        lo, hi = max(0, -s), min(L, L - s)
        if lo < hi:
            z[:, lo:hi, :] += x[:, lo + s:hi + s, :] @ w[t]
    return z


def forward(params, feats, lengths, bf16: bool = False):
    layers = unpack(params)
    B, L, _ = feats.shape
    m = _mask(B, L, lengths)[:, :, None]
    x = np.asarray(feats, dtype=np.float64) * m
    cache = []
    for li, (w, b) in enumerate(layers):
        if bf16:
            x = bf16_round(x)
            w = bf16_round(w)
        z = (_conv(x, w) + b) * m
        cache.append((x, w, z))
        x = np.maximum(z, 0.0) if li < len(layers) - 1 else z
    return x, cache


def loss_and_grad(params, feats, targets, lengths, bf16: bool = False):
    """Mean squared error and its gradient w.r.t. the flat parameters."""
    y, cache = forward(params, feats, lengths, bf16)
    B, L, _ = feats.shape
    m = _mask(B, L, lengths)[:, :, None]
    cnt = float(m.sum()) * y.shape[2]
    r = (y - np.asarray(targets, dtype=np.float64)) * m
    loss = float((r * r).sum() / cnt)
    dz = 2.0 * r / cnt
    grads = []
    for li in range(len(cache) - 1, -1, -1):
        x, w, z = cache[li]
        dw = np.zeros_like(w)
        for t in range(TAPS):
            s = t - 2
            lo, hi = max(0, -s), min(L, L - s)
            if lo < hi:
                dw[t] = np.einsum("blc,bld->cd", x[:, lo + s:hi + s, :], dz[:, lo:hi, :])
        db = dz.sum(axis=(0, 1))
        grads.append((dw, db))
        if li > 0:
            dx = np.zeros_like(x)
            for t in range(TAPS):
                s = t - 2
                lo, hi = max(0, -s), min(L, L - s)
                if lo < hi:
                    dx[:, lo + s:hi + s, :] += dz[:, lo:hi, :] @ w[t].T
            prev_z = cache[li - 1][2]
            dz = dx * (prev_z > 0) * m
    grads.reverse()
    flat = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    return loss, flat
