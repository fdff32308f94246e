"""Plain FP64 numpy U-Net -- TEST INFRASTRUCTURE ONLY.

The reference for the surrogate's CUDA kernels: the same 4-level U-Net
(3 x 3 convolutions with ReLU, 2 x 2 average pooling, nearest 2x upsampling,
[upsampled, skip] concatenation, 1 x 1 head) written as the textbook
definitions, with the backward pass derived by hand layer by layer.  Arrays
are [B][C][H][W].  Only tests use it.
"""
from __future__ import annotations

import numpy as np


def exact(a):
    return a


def bf16(a):
    """Round to BF16 (8 significant bits, nearest even) by way of FP32, the
    storage type of the values a BF16 product is formed from; returned as
    FP64.  Passed as `rnd` below, it makes every product's operands BF16
    while sums stay FP64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def conv(x, w, b, relu, rnd=exact):
    """Cross-correlation with zero padding (k - 1) / 2, stride 1:
    y[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, i + u - p, j + v - p].
    rnd: applied to both factors of the products (w and x)."""
    k = w.shape[2]
    p = (k - 1) // 2
    w = rnd(w)
    xp = np.pad(rnd(x), ((0, 0), (0, 0), (p, p), (p, p)))
    H, W = x.shape[2], x.shape[3]
    y = np.zeros((x.shape[0], w.shape[0], H, W))
    for u in range(k):
        for v in range(k):
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], xp[:, :, u:u + H, v:v + W])
    y += b[None, :, None, None]
    return np.maximum(y, 0.0) if relu else y


def conv_backward(x, w, y, dy, relu, rnd=exact):
    """Gradients of conv() with respect to x, w and b, given dL/dy; rnd is
    applied to the factors of every product (dy and x for dw, w and dy for dx)."""
    if relu:
        dy = dy * (y > 0)
    k = w.shape[2]
    p = (k - 1) // 2
    H, W = x.shape[2], x.shape[3]
    xp = np.pad(rnd(x), ((0, 0), (0, 0), (p, p), (p, p)))
    dyr, wr = rnd(dy), rnd(w)
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for u in range(k):
        for v in range(k):
            dw[:, :, u, v] = np.einsum("nohw,nchw->oc", dyr, xp[:, :, u:u + H, v:v + W])
            dxp[:, :, u:u + H, v:v + W] += np.einsum("oc,nohw->nchw", wr[:, :, u, v], dyr)
    dx = dxp[:, :, p:p + H, p:p + W]
    return dx, dw, dy.sum(axis=(0, 2, 3))


def pool(x):
    return 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 1::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 1::2])


def pool_backward(dy):
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_backward(dy):
    return dy[:, :, 0::2, 0::2] + dy[:, :, 1::2, 0::2] + dy[:, :, 0::2, 1::2] + dy[:, :, 1::2, 1::2]


def forward(params, x, rnd=exact):
    """Returns the output and the cache of every layer's input and output."""
    P = params
    cache = {}

    def layer(name, inp, relu=True):
        out = conv(inp, P[name + ".w"], P[name + ".b"], relu, rnd)
        cache[name] = (inp, out, relu)
        return out

    s1 = layer("enc1b", layer("enc1a", x))
    s2 = layer("enc2b", layer("enc2a", pool(s1)))
    s3 = layer("enc3b", layer("enc3a", pool(s2)))
    bt = layer("botb", layer("bota", pool(s3)))
    d3 = layer("dec3b", layer("dec3a", np.concatenate([up(bt), s3], axis=1)))
    d2 = layer("dec2b", layer("dec2a", np.concatenate([up(d3), s2], axis=1)))
    d1 = layer("dec1b", layer("dec1a", np.concatenate([up(d2), s1], axis=1)))
    out = layer("head", d1, relu=False)
    return out, cache


def backward(params, cache, dout, rnd=exact):
    """Gradients of every parameter given dL/dout (same keys as params)."""
    g = {}

    def back(name, dy):
        inp, out, relu = cache[name]
        dx, dw, db = conv_backward(inp, params[name + ".w"], out, dy, relu, rnd)
        g[name + ".w"], g[name + ".b"] = dw, db
        return dx

    def split(dcat, c_up):
        return dcat[:, :c_up], dcat[:, c_up:]

    dd1 = back("head", dout)
    dcat1 = back("dec1a", back("dec1b", dd1))
    c_up = cache["dec1a"][0].shape[1] - cache["enc1b"][1].shape[1]
    dup2, ds1 = split(dcat1, c_up)
    dcat2 = back("dec2a", back("dec2b", up_backward(dup2)))
    c_up = cache["dec2a"][0].shape[1] - cache["enc2b"][1].shape[1]
    dup3, ds2 = split(dcat2, c_up)
    dcat3 = back("dec3a", back("dec3b", up_backward(dup3)))
    c_up = cache["dec3a"][0].shape[1] - cache["enc3b"][1].shape[1]
    dupb, ds3 = split(dcat3, c_up)
    dbt = up_backward(dupb)
    ds3 = ds3 + pool_backward(back("bota", back("botb", dbt)))
    ds2 = ds2 + pool_backward(back("enc3a", back("enc3b", ds3)))
    ds1 = ds1 + pool_backward(back("enc2a", back("enc2b", ds2)))
    back("enc1a", back("enc1b", ds1))
    return g


def mse(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size
