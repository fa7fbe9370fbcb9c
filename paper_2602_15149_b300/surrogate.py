"""Learned constitutive surrogate of the J2 return map: data generation, training, evaluation.

Every computation runs in the library (tlsph_j2_samples, tlsph_mlp_*); this module only
orders the calls.  torch provides the device buffers and the shuffled batch order.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import tlsph


def he_uniform(seed=0, sizes=(16, 128, 128, 128, 16)):
    rng = np.random.default_rng(seed)
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = math.sqrt(6.0 / n_in)
        params.append((rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)))
    return tlsph.pack_params(params)


def generate_samples(case, n_target, steps, every=20, stride_elastic=4, stride_plastic=1, device=0, stream=None,
                     precision=None, per_call=None):
    """Run the workload with the exact return map and collect (x, y, |P|) rows every `every` steps.

    With `per_call`, both strides double after a call that kept more rows than that, so that the
    samples spread over the whole run instead of filling up in its first steps."""
    import torch

    dev = torch.device("cuda", device)
    x = torch.empty((n_target, 16), dtype=torch.float32, device=dev)
    y = torch.empty((n_target, 16), dtype=torch.float32, device=dev)
    pn = torch.empty((n_target,), dtype=torch.float32, device=dev)
    g = tlsph.from_case(case, precision=precision, device=device, stream=stream)
    n, k, salt = 0, 0, 0
    while k < steps and n < n_target:
        g.step(every)
        k += every
        salt += 1
        got = g.j2_samples(x[n:], y[n:], stride_elastic, stride_plastic, salt, pnorm=pn[n:])
        n += got
        if per_call and got > per_call:
            stride_elastic, stride_plastic = 2 * stride_elastic, 2 * stride_plastic
    g.close()
    return x[:n], y[:n], pn[:n]


def train(x, y, epochs=10, batch=4096, lr=2e-3, lr_end=1e-5, seed=0, device=0, time_budget_s=None, log=None):
    """Train a fresh network on (x, y) with Adam and a cosine learning-rate schedule.

    With a time budget the number of epochs is cut after the first one to what fits, and the
    schedule is stretched over the epochs that remain, so it still ends at lr_end."""
    import torch

    mlp = tlsph.MLP(batch=batch, device=device)
    mlp.set_params(he_uniform(seed))
    mlp.fit_normalization(x, y, margin=0.0)
    n = x.shape[0]
    nb = n // batch
    total = max(1, epochs * nb)
    gen = torch.Generator(device=x.device).manual_seed(seed)
    t0 = time.perf_counter()
    step, losses = 0, []
    ep = 0
    while ep < epochs:
        perm = torch.randperm(n, device=x.device, generator=gen)
        xs, ys = x.index_select(0, perm), y.index_select(0, perm)
        for b in range(nb):
            a = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * min(step, total) / total))
            loss = mlp.train_step(xs[b * batch:(b + 1) * batch], ys[b * batch:(b + 1) * batch], a)
            step += 1
        losses.append(loss)
        ep += 1
        elapsed = time.perf_counter() - t0
        if log:
            log(f"epoch {ep}: loss {loss:.3e} ({elapsed:.1f} s)")
        if time_budget_s and ep == 1 and epochs > 1:
            epochs = max(1, min(epochs, int(time_budget_s / max(elapsed, 1e-9))))
            total = max(1, epochs * nb)
    return mlp, {"epochs": len(losses), "steps": step, "final_loss": losses[-1] if losses else None,
                 "train_s": time.perf_counter() - t0, "samples": n}


def stress_error(mlp, x, y, pnorm, sigma_y0):
    """Per-sample relative stress error |P_net - P_exact|_F / max(|P_exact|_F, sigma_y0) (mean, p99,
    max) over the rows inside the envelope.  The stress columns of y hold P - P^tr, the network's
    as well, so their difference is P_net - P_exact."""
    import torch

    out = torch.empty_like(y)
    outside = torch.zeros(x.shape[0], dtype=torch.int32, device=x.device)
    mlp.forward(x, out, outside)
    inside = outside == 0
    d = torch.linalg.norm(out[:, :9] - y[:, :9], dim=1)
    ref = torch.clamp(pnorm, min=sigma_y0)
    e = (d / ref)[inside].double()
    return {"mean": float(e.mean()), "p99": float(torch.quantile(e.float(), 0.99)), "max": float(e.max()),
            "inside_fraction": float(inside.float().mean())}
