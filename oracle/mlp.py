"""Neural materials oracle (TEST INFRASTRUCTURE): positional encoding + MLP in
numpy FP64, with BF16 round-to-nearest-even applied exactly where the GPU keeps
values in BF16 (weights and the input of every layer).

Paper (arXiv 2311.18558, Sec. III-D, Eq. pos_encoding): the scene coordinates are
normalised to the unit cube, p_bar = (p - b) / Delta_b (b the centre and Delta_b
the size of the scene's bounding box), encoded per coordinate as
gamma(p) = [sin(2 pi p), cos(2 pi p), ..., sin(2^L pi p), cos(2^L pi p)], fed to an
MLP whose outputs are transformed as in Eq. trainable_materials_1/2:
sigma = exp(o_1), eps_r = 1 + exp(o_2).

Readings: Delta_b is the longest edge of the bounding box; the encoding is
prefixed by p_bar itself (3 + 6L features, 39 for L = 6), in the order
[p_bar, then for k = 1..L: sin(2^k pi p_bar_x,y,z), cos(2^k pi p_bar_x,y,z)];
the MLP is evaluated at triangle centroids, hidden layers use ReLU.
"""
from __future__ import annotations

import numpy as np

L_FREQ = 6
D_IN = 3 + 6 * L_FREQ


def bf16_round(x):
    """Round float values to the nearest BF16 (ties to even), returned as float64.

    BF16 keeps the top 16 bits of the IEEE FP32 pattern; rounding to nearest even
    adds 0x7FFF plus the lowest kept bit before truncating the low 16 bits."""
    f = np.asarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def normalize(points, lo, hi):
    """p_bar = (p - b) / Delta_b, b the box centre, Delta_b its longest edge."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return (np.asarray(points, np.float64) - 0.5 * (lo + hi)) / np.max(hi - lo)


def encode(pbar, L=L_FREQ):
    """[p_bar, sin(2^k pi p_bar), cos(2^k pi p_bar) for k = 1..L] (Eq. pos_encoding)."""
    feats = [pbar]
    for k in range(1, L + 1):
        w = (2.0 ** k) * np.pi
        feats.append(np.sin(w * pbar))
        feats.append(np.cos(w * pbar))
    return np.concatenate(feats, axis=1)


def forward(x, Ws, bs, bf16=True):
    """MLP forward.  Returns (output (n, 2), list of layer inputs, list of pre-activations)."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    a = rnd(x)
    ins, pre = [], []
    for i, (W, b) in enumerate(zip(Ws, bs)):
        ins.append(a)
        z = a @ rnd(W) + np.asarray(b, np.float64)
        pre.append(z)
        if i < len(Ws) - 1:
            a = rnd(np.maximum(z, 0.0))
        else:
            a = z
    return a, ins, pre


def materials(out):
    """sigma = exp(o_1), eps_r = 1 + exp(o_2) (Eq. trainable_materials_1/2)."""
    return 1.0 + np.exp(out[:, 1]), np.exp(out[:, 0])


def backward(x, Ws, bs, grad_eps, grad_sigma, bf16=True):
    """Gradients of L w.r.t. every weight and bias given dL/deps_r and dL/dsigma per
    point; weights enter as their BF16 values, gradients are kept in FP64."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    out, ins, pre = forward(x, Ws, bs, bf16)
    eps, sig = materials(out)
    g = np.stack([np.asarray(grad_sigma, np.float64) * sig, np.asarray(grad_eps, np.float64) * (eps - 1.0)], 1)
    gW = [None] * len(Ws)
    gb = [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        gW[i] = ins[i].T @ g
        gb[i] = g.sum(axis=0)
        if i > 0:
            g = (g @ rnd(Ws[i]).T) * (pre[i - 1] > 0)
    return gW, gb
