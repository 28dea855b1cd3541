"""Subspace network: a plain multilayer perceptron, forward, backward, Adam.

The paper has no learned component; this module is the float64 oracle for
the network that predicts a vertex's basis U_i (see ``learned``).

Architecture: widths ``dims = [d_in, h, ..., h, d_out]``; every hidden layer
is ``H_l = GELU(H_{l-1} W_l^T + b_l)`` with the erf form of GELU,
``GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2`` (Hendrycks and Gimpel,
2016); the output layer is linear.  Loss: mean squared error over all
``B * d_out`` outputs.  Optimiser: Adam (Kingma and Ba, 2015, Algorithm 1)
with bias correction.

Parameters are one flat vector, layer by layer: ``W_l`` row-major
``[dims[l+1], dims[l]]``, then ``b_l`` ``[dims[l+1]]``.

Rounding.  With ``rounding=True`` the computation rounds to bfloat16 at the
points where the tensor-core path stores bfloat16 operands: the input X,
every weight matrix, every hidden activation H_l, the output gradient dY and
every pre-activation gradient dZ_l.  Everything else (products, sums, GELU,
biases, the loss) is float64 here; the GPU accumulates in float32.  With
``rounding=False`` the whole computation is plain float64 (used by the
finite-difference pins).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np
from scipy.special import erf


def bf16(a) -> np.ndarray:
    """Round to bfloat16 as the GPU stores values: float64 -> float32 (nearest,
    ties to even), then float32 -> bfloat16 by rounding away the low 16 bits
    of the float32 pattern to nearest, ties to even.  Returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (r.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def gelu(z: np.ndarray) -> np.ndarray:
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def layer_slices(dims: List[int]) -> List[Tuple[slice, slice]]:
    """(weight slice, bias slice) of every layer in the flat parameter vector."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        out.append((slice(o, o + nw), slice(o + nw, o + nw + dims[l + 1])))
        o += nw + dims[l + 1]
    return out


def unpack(params: np.ndarray, dims: List[int]):
    p = np.asarray(params, dtype=np.float64)
    return [(p[sw].reshape(dims[l + 1], dims[l]), p[sb]) for l, (sw, sb) in enumerate(layer_slices(dims))]


def forward(params, dims: List[int], X, rounding: bool = True):
    """Y [B, d_out] and the cache (layer inputs H_l, pre-activations Z_l)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params, dims)
    H = r(X)
    inputs, pre = [], []
    for l, (W, b) in enumerate(layers):
        inputs.append(H)
        Z = H @ r(W).T + b
        pre.append(Z)
        if l < len(layers) - 1:
            H = r(gelu(Z))
    return Z, (inputs, pre)


def loss_and_grad(params, dims: List[int], X, T, rounding: bool = True):
    """Mean squared error and its gradient (flat, parameter layout)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params, dims)
    Y, (inputs, pre) = forward(params, dims, X, rounding)
    T = np.asarray(T, dtype=np.float64)
    B, d_out = Y.shape
    diff = Y - T
    loss = float(np.sum(diff * diff) / (B * d_out))
    grad = np.zeros(len(params))
    slices = layer_slices(dims)
    dZ = r(2.0 * diff / (B * d_out))
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        sw, sb = slices[l]
        grad[sw] = (dZ.T @ inputs[l]).ravel()
        grad[sb] = dZ.sum(axis=0)
        if l > 0:
            dH = dZ @ r(W)
            dZ = r(dH * gelu_grad(pre[l - 1]))
    return loss, grad


def adam_step(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step number t >= 1): returns (params, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p = np.asarray(params, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v
