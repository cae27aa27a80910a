"""CPU FP64 reference of the learned warm start's network. TEST INFRASTRUCTURE.

Only the tests and the benchmark's CPU-baseline leg use this module.  The
network is a plain multilayer perceptron (the paper has no learned part;
this is the warm-start model the GPU trains): features -> three hidden
layers with GELU (tanh form) -> linear output, mean squared error against
the labels.  Forward and backward are written out layer by layer in
float64 numpy; the backward pass is pinned by central finite differences in
the tests.  Where the GPU keeps a tensor in bf16, callers round with
`bf16` at the same points.
"""
from __future__ import annotations

import numpy as np

_K0 = 0.7978845608028654
_K1 = 0.044715


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_K0 * (x + _K1 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(_K0 * (x + _K1 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _K0 * (1.0 + 3.0 * _K1 * x * x)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X, round_bf16=False):
    """params: list of (W [out, in], b [out]); returns (Y, cache)."""
    cache = []
    H = bf16(X) if round_bf16 else X
    for li, (W, b) in enumerate(params):
        Wr = bf16(W) if round_bf16 else W
        Z = H @ Wr.T + b
        cache.append((H, Z))
        if li < len(params) - 1:
            H = gelu(Z)
            if round_bf16:
                H = bf16(H)
        else:
            H = Z
    return H, cache


def loss_and_grads(params, X, T, n_out, round_bf16=False, magnitudes=False):
    """Mean squared error over the first n_out outputs and its gradients.

    With magnitudes=True it also returns, per layer, the sums of the
    absolute values of the terms that make up each gradient entry
    (|g|^T |H| for the weights, sum |g| for the biases): the scale against
    which a rounding difference in one of those terms is measured."""
    Y, cache = forward(params, X, round_bf16)
    B = X.shape[0]
    D = np.zeros_like(Y)
    D[:, :n_out] = Y[:, :n_out] - T
    loss = float(np.sum(D ** 2) / (B * n_out))
    dY = 2.0 * D / (B * n_out)
    grads = [None] * len(params)
    mags = [None] * len(params)
    g = dY                      # gradient w.r.t. this layer's pre-activation
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        H, Z = cache[li]
        if li < len(params) - 1:
            g = g * gelu_grad(Z)
        g16 = bf16(g) if round_bf16 else g     # operand of the weight and input GEMMs
        Wr = bf16(W) if round_bf16 else W
        grads[li] = (g16.T @ H, g.sum(axis=0))
        if magnitudes:
            mags[li] = (np.abs(g16).T @ np.abs(H), np.abs(g).sum(axis=0))
        g = g16 @ Wr
    if magnitudes:
        return loss, grads, mags
    return loss, grads
