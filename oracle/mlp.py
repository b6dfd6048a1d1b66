"""FP64 oracle of the initial-guess MLP (TEST INFRASTRUCTURE ONLY).

Only tests/, the smoke check and the benchmark's CPU-baseline leg import this
module; it shares no code with the CUDA library.

The network (an extension of the solver, not in the paper): inputs are a
system's diagonal, right-hand side and previous solution (3n values,
standardised), three hidden layers with GELU (tanh form), and a linear output
of n values (the standardised change of the solution). Loss: mean squared
error over all outputs of a minibatch. Optimiser: Adam (Kingma & Ba).

Parameters are a list of (W, b) per layer with W of shape [out, in]
(y = x W^T + b). With `round_bf16=True` the forward pass rounds the layer
inputs, weights and hidden activations to bfloat16 (round to nearest even)
where the GPU stores them in bfloat16, and the backward pass rounds the
activation gradients likewise; arithmetic stays FP64.

Pinned by: central finite differences of the loss (gradients), zero weights
(output = bias), GELU values at fixed points, one Adam step against its
closed form (tests/test_oracle_mlp.py).
"""

from __future__ import annotations

import numpy as np

SQRT_2_OVER_PI = np.sqrt(2.0 / np.pi)
GELU_C = 0.044715


def to_bf16(a):
    """Round an array to the nearest bfloat16 value (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def gelu(z):
    """GELU, tanh form: 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(SQRT_2_OVER_PI * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    u = SQRT_2_OVER_PI * (z + GELU_C * z ** 3)
    t = np.tanh(u)
    du = SQRT_2_OVER_PI * (1.0 + 3.0 * GELU_C * z ** 2)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def init_params(sizes, rng):
    """He-style uniform init for layers sizes[0] -> sizes[1] -> ... (tests only)."""
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / fan_in) * 0.5
        params.append((rng.uniform(-bound, bound, (fan_out, fan_in)), rng.uniform(-0.1, 0.1, fan_out)))
    return params


def forward(params, X, round_bf16=False):
    """Returns (out, cache). Hidden layers use GELU; the last layer is linear."""
    r = to_bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = r(X)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        Wl = r(W)
        z = h @ Wl.T + b
        cache.append((h, Wl, z))
        if l < L - 1:
            h = r(gelu(z))
        else:
            h = z
    return h, cache


def loss_and_grads(params, X, Y, round_bf16=False):
    """MSE loss mean((out - Y)^2) over all elements and its parameter gradients."""
    out, cache = forward(params, X, round_bf16)
    M, n = out.shape
    diff = out - Y
    loss = float(np.mean(diff * diff))
    r = to_bf16 if round_bf16 else (lambda a: a)
    d = r(2.0 * diff / (M * n))
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h, Wl, z = cache[l]
        if l < len(params) - 1:
            d = r(d * gelu_grad(z))
        gW = d.T @ h
        gb = d.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            d = d @ Wl
    return loss, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; state is (t, m, v) with m, v lists like params."""
    t, m, v = state
    t += 1
    new_params, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mhat = mm / (1 - beta1 ** t)
            vhat = vv / (1 - beta2 ** t)
            out.append((p - lr * mhat / (np.sqrt(vhat) + eps), mm, vv))
        new_params.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_params, (t, new_m, new_v)


def zero_state(params):
    z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    return (0, z, [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat, sizes):
    params, o = [], 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + fan_in * fan_out].reshape(fan_out, fan_in)
        o += fan_in * fan_out
        b = flat[o:o + fan_out]
        o += fan_out
        params.append((np.array(W, dtype=np.float64), np.array(b, dtype=np.float64)))
    return params
