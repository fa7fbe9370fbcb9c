"""Pins of the FP64 reference network (oracle/mlp.py): finite differences and closed forms."""
import numpy as np

from oracle import mlp


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 101)
    assert np.allclose(mlp.silu(z), z * 0.5 * (1 + np.tanh(z / 2)), rtol=1e-14, atol=1e-15)
    e = 1e-6
    fd = (mlp.silu(z + e) - mlp.silu(z - e)) / (2 * e)
    assert np.abs(fd - mlp.silu_grad(z)).max() < 1e-8


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(seed=1)
    x = rng.normal(size=(7, 16))
    y = rng.normal(size=(7, 16))
    loss, grads = mlp.loss_and_grads(p, x, y)
    e = 1e-6
    for l in range(4):
        W, b = p[l]
        for _ in range(4):
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += e
            Wm[i, j] -= e
            pp = [(Wp, b) if k == l else p[k] for k in range(4)]
            pm = [(Wm, b) if k == l else p[k] for k in range(4)]
            fd = (mlp.loss_and_grads(pp, x, y)[0] - mlp.loss_and_grads(pm, x, y)[0]) / (2 * e)
            assert abs(fd - grads[l][0][i, j]) <= 1e-6 * max(1.0, abs(fd))
        k = rng.integers(b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[k] += e
        bm[k] -= e
        pp = [(W, bp) if q == l else p[q] for q in range(4)]
        pm = [(W, bm) if q == l else p[q] for q in range(4)]
        fd = (mlp.loss_and_grads(pp, x, y)[0] - mlp.loss_and_grads(pm, x, y)[0]) / (2 * e)
        assert abs(fd - grads[l][1][k]) <= 1e-6 * max(1.0, abs(fd))


def test_linear_limit():
    """With every hidden pre-activation tiny, SiLU(z) ~ z/2: the network is the product of the layers / 8."""
    p = mlp.init_params(seed=2)
    p = [(W * 1e-3 if l < 3 else W, b) for l, (W, b) in enumerate(p)]
    x = np.random.default_rng(3).normal(size=(5, 16)) * 1e-3
    out, _ = mlp.forward(p, x)
    lin = x
    for l, (W, b) in enumerate(p):
        lin = lin @ W.T + b
        if l < 3:
            lin = lin / 2
    assert np.abs(out - lin).max() <= 1e-4 * np.abs(lin).max()
