"""FP64 reference of the constitutive surrogate network (test infrastructure only).

The surrogate is a multilayer perceptron 16 -> 128 -> 128 -> 128 -> 16 with SiLU
activations after the three hidden layers and a linear output.  Layer l maps
a row vector x to z = x W_l^T + b_l (W_l has shape out x in).  The loss of a batch
is the mean over the batch of the squared error summed over the 16 outputs,
divided by 16 (the mean squared error).  This module writes the forward and the
backward pass out plainly (numpy FP64); the device kernels are checked against it.
"""
from __future__ import annotations

import numpy as np

SIZES = (16, 128, 128, 128, 16)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed=0, sizes=SIZES):
    """He-style uniform initialisation; returns [(W0, b0), ...] in FP64."""
    rng = np.random.default_rng(seed)
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / n_in)
        params.append((rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)))
    return params


def forward(params, x):
    """Return the output and the list of (input, pre-activation) of every layer."""
    cache = []
    a = np.asarray(x, dtype=np.float64)
    for l, (W, b) in enumerate(params):
        z = a @ W.T + b
        cache.append((a, z))
        a = silu(z) if l < len(params) - 1 else z
    return a, cache


def loss_and_grads(params, x, y):
    """Mean squared error of a batch and its gradient with respect to every W, b."""
    out, cache = forward(params, x)
    B, m = out.shape
    err = out - y
    loss = float(np.sum(err * err) / (B * m))
    d = 2.0 * err / (B * m)  # dL/d(output)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        a_in, z = cache[l]
        if l < len(params) - 1:
            d = d * silu_grad(z)  # through the activation of layer l
        W, _ = params[l]
        grads[l] = (d.T @ a_in, d.sum(axis=0))
        d = d @ W
    return loss, grads
