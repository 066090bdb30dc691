"""CPU oracle of the surrogate network (include/lbib_mlp.h): plain numpy, FP64.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/`` and ``bench.py``'s
CPU-baseline leg may import it.  It shares no code with the CUDA library.

The network and its training loss are stated in include/lbib_mlp.h:
  a_0 = s_in (x - c_in),  z_l = W_l a_{l-1} + b_l,  a_l = GELU(z_l),
  y_raw = W_out a_H + b_out,  y = s_out y_raw + c_out,
  loss = mean over batch and outputs of (y_raw - (t - c_out) / s_out)^2,
GELU in its tanh form (Hendrycks & Gimpel 2016),
  GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
which lies within 5e-4 of z Phi(z).  ``forward`` / ``gradients`` with
quantize=False are that definition in FP64 (matrix products by numpy; the backward pass is the chain
rule written out layer by layer) and are pinned by finite differences in
tests/test_oracle_mlp.py.  quantize=True inserts the library's roundings at
the same points: weights and activations to bfloat16 (round to nearest even),
the input scaling and the targets' standardisation in float32, the output
gradient and the back-propagated pre-activation gradients to bfloat16; the
products stay exact (FP64) where the GPU accumulates in FP32.  ``adam_step`` is
the optimiser's update rule; it is pinned by its closed forms (first step and
constant gradient move every parameter by lr against the gradient's sign).
"""
from __future__ import annotations

import math

import numpy as np


def bf16(x) -> np.ndarray:
    """float32 values rounded to bfloat16 (round to nearest, ties to even),
    returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)
GELU_CUBIC = 0.044715


def _gelu_tanh(z):
    return np.tanh(SQRT_2_OVER_PI * (z + GELU_CUBIC * z ** 3))


def gelu(z):
    """GELU in the tanh form of Hendrycks & Gimpel (Gaussian Error Linear
    Units, 2016): z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + _gelu_tanh(z))


def gelu_d(z):
    """d gelu / dz: (1 + t)/2 + z/2 (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2),
    t the tanh of gelu."""
    z = np.asarray(z, np.float64)
    t = _gelu_tanh(z)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * SQRT_2_OVER_PI * (1.0 + 3.0 * GELU_CUBIC * z * z)


def split_params(p, n_in, width, n_hidden, n_out):
    """[(W, b), ...] in the library's flat order (hidden layers, then output)."""
    dims = [n_in] + [width] * n_hidden + [n_out]
    out, k = [], 0
    for i, o in zip(dims[:-1], dims[1:]):
        W = np.asarray(p[k:k + o * i], np.float64).reshape(o, i)
        k += o * i
        b = np.asarray(p[k:k + o], np.float64)
        k += o
        out.append((W, b))
    return out


def _q(v, on):
    return bf16(v) if on else np.asarray(v, np.float64)


def forward(layers, x, c_in, s_in, c_out, s_out, quantize=False):
    """Returns y (physical units), y_raw, and the per-layer (a_in, z) cache."""
    if quantize:
        a = bf16(np.float32(s_in) * (np.asarray(x, np.float32) - np.float32(c_in)))
    else:
        a = np.asarray(s_in, np.float64) * (np.asarray(x, np.float64) - np.asarray(c_in, np.float64))
    cache = []
    for W, b in layers[:-1]:
        z = a @ _q(W, quantize).T + b
        cache.append((a, z))
        a = _q(gelu(z), quantize)
    W, b = layers[-1]
    yraw = a @ _q(W, quantize).T + b
    cache.append((a, None))
    y = np.asarray(s_out, np.float64) * yraw + np.asarray(c_out, np.float64)
    return y, yraw, cache


def gradients(layers, x, t, c_in, s_in, c_out, s_out, quantize=False):
    """Loss and [(dW, db), ...] by the chain rule, layer by layer."""
    _, yraw, cache = forward(layers, x, c_in, s_in, c_out, s_out, quantize)
    B, n_out = yraw.shape
    if quantize:
        ts = (np.asarray(t, np.float32) - np.float32(c_out)) / np.float32(s_out)
    else:
        ts = (np.asarray(t, np.float64) - np.asarray(c_out, np.float64)) / np.asarray(s_out, np.float64)
    d = yraw - ts
    loss = float(np.mean(d * d))
    g = _q(2.0 * d / (B * n_out), quantize)  # d loss / d y_raw
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        a_in, _ = cache[l]
        grads[l] = (g.T @ a_in, g.sum(axis=0))
        if l == 0:
            break
        W, _ = layers[l]
        _, z_prev = cache[l - 1]
        g = _q((g @ _q(W, quantize)) * gelu_d(z_prev), quantize)
    return loss, grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in FP64: moment
    estimates m, v updated with gradient g at step t (1-based), bias-corrected,
    p moved by lr * m_hat / (sqrt(v_hat) + eps).  Returns (p, m, v)."""
    p, g = np.asarray(p, np.float64), np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def flat(grads) -> np.ndarray:
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
