"""FP64 CPU reference of the warm-start MLP (test infrastructure only).

y = W3 g(W2 g(W1 x + b1) + b2) + b3, g(z) = z Phi(z) (GELU, erf form), loss =
mean over all outputs of (y - t)^2.  Plain numpy, written from these
definitions; the backward pass is the chain rule layer by layer.  Optionally
rounds weights and layer inputs to BF16 (round-to-nearest-even) the way the
GPU kernels feed their tensor-core products, so both sides can be compared
tightly.  Pinned by finite differences in the tests.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params: dict, x: np.ndarray, bf16: bool = False):
    """Returns (y, cache).  params: W1 (h,in), b1, W2 (h,h), b2, W3 (out,h), b3."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = r(params["W1"]), r(params["W2"]), r(params["W3"])
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    x0 = r(x)
    z1 = x0 @ W1.T + b1
    a1 = r(gelu(z1))
    z2 = a1 @ W2.T + b2
    a2 = r(gelu(z2))
    y = a2 @ W3.T + b3
    return y, dict(x0=x0, z1=z1, a1=a1, z2=z2, a2=a2, W1=W1, W2=W2, W3=W3)


def loss_and_grads(params: dict, x: np.ndarray, t: np.ndarray, bf16: bool = False):
    """MSE loss and its gradient with respect to every parameter (chain rule)."""
    y, c = forward(params, x, bf16)
    n = y.size
    d = y - np.asarray(t, np.float64)
    loss = float(np.sum(d * d) / n)
    r = bf16_round if bf16 else (lambda a: a)
    dy = 2.0 * d / n
    dyr = r(dy)
    g = {}
    g["W3"] = dyr.T @ c["a2"]
    g["b3"] = dy.sum(axis=0)
    da2 = dyr @ c["W3"]
    dz2 = da2 * gelu_grad(c["z2"])
    dz2r = r(dz2)
    g["W2"] = dz2r.T @ c["a1"]
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2r @ c["W2"]
    dz1 = da1 * gelu_grad(c["z1"])
    dz1r = r(dz1)
    g["W1"] = dz1r.T @ c["x0"]
    g["b1"] = dz1.sum(axis=0)
    return loss, g
