"""Plain NumPy FP64 multilayer perceptron: the oracle for the surrogate's tensor-core MLP kernels.

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``).

x -> relu(W_0 x + b_0) -> ... -> W_{L-1} h + b_{L-1};
loss = sum_b r_b sum_j w_j (y_bj - t_bj)^2 / (B n_out), with per-output weights w (wmask) and
per-sample weights r (rowweight), both 1 when not given.
With ``bf16=True`` the values the library stores in bfloat16 are rounded the same way (round to
nearest even): weights to bf16; every layer input (features and hidden activations) to the split
pair bf16(a) + bf16(a - bf16(a)); output and hidden gradients to bf16.  The comparison then isolates
accumulation order.  With ``bf16=False`` it is exact FP64 backpropagation, pinned against central
finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) through float32, returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split(x: np.ndarray) -> np.ndarray:
    """The library's split-precision layer input: bf16(x) + bf16(x - bf16(x)) (FP32 differences)."""
    hi = bf16(x)
    lo = bf16(np.asarray(x, dtype=np.float32).astype(np.float64) - hi)
    return hi + lo


def unpack(params: np.ndarray, layout):
    """Split the library's padded FP32 parameter vector into [(W, b)] (FP64)."""
    out = []
    for woff, o, i, boff in layout:
        W = params[woff:woff + o * i].astype(np.float64).reshape(o, i)
        b = params[boff:boff + o].astype(np.float64)
        out.append((W, b))
    return out


def forward(layers, X, bf=True):
    """Returns (y, cache) for a batch X [B, n_in_padded]."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    sp = split if bf else (lambda v: np.asarray(v, dtype=np.float64))
    h = sp(X)
    cache = [h]
    pres = []
    for li, (W, b) in enumerate(layers):
        pre = h @ r(W).T + b
        pres.append(pre)
        if li + 1 < len(layers):
            h = sp(np.maximum(pre, 0.0).astype(np.float32) if bf else np.maximum(pre, 0.0))
            cache.append(h)
        else:
            h = pre
    return h, (cache, pres)


def loss_and_grads(layers, X, T, nout, wmask=None, bf=True, rowweight=None):
    """Weighted MSE loss over the first nout outputs and the gradients [(dW, db)] (same shapes as
    layers); wmask weights the outputs, rowweight the samples."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    y, (acts, pres) = forward(layers, X, bf)
    B = X.shape[0]
    w = np.ones(nout) if wmask is None else np.asarray(wmask, dtype=np.float64)
    r_b = np.ones(B) if rowweight is None else np.asarray(rowweight, dtype=np.float64)
    d = y[:, :nout] - T[:, :nout]
    loss = float((r_b[:, None] * w * d * d).sum() / (B * nout))
    g = np.zeros_like(y)
    g[:, :nout] = 2.0 * r_b[:, None] * w * d / (B * nout)
    g = r(g)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (g.T @ acts[li], g.sum(axis=0))
        if li == 0:
            break
        dA = g @ r(W)
        g = r(dA * (pres[li - 1] > 0))
    return loss, grads
