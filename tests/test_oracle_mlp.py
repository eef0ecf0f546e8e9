"""Pins of the CPU reference network used to check the GPU training kernels.

The manual backward pass must equal central finite differences of the loss
(the gradient is then pinned by the loss alone, which is a plain sum), and
the network must be exactly odd in T.
"""
import numpy as np

from oracle import mlp_ref


def _setup(seed=0, n=16):
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=0.3, size=mlp_ref.N_PARAMS)
    T = rng.normal(size=(n, 3))
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    y = rng.normal(scale=0.05, size=(n, 27))
    scale = rng.uniform(0.02, 0.1, 27)
    return theta, T, y, scale


def test_param_count():
    assert mlp_ref.N_PARAMS == 128 * 3 + 128 + 2 * (128 * 128 + 128) + 32 * 128 + 32 == 37664


def test_backward_matches_finite_differences():
    theta, T, y, scale = _setup()
    _, g = mlp_ref.loss_and_grad(theta, T, y, scale)
    rng = np.random.default_rng(1)
    # every parameter block, plus random entries; W4 rows 27..31 have zero gradient
    idx = list(rng.choice(mlp_ref.N_PARAMS, 60, replace=False))
    o = 0
    for name, shp in mlp_ref.SIZES:
        idx.append(o)
        o += int(np.prod(shp))
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (mlp_ref.loss_only(tp, T, y, scale) - mlp_ref.loss_only(tm, T, y, scale)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_network_is_odd():
    theta, T, y, scale = _setup(2)
    h1, _ = mlp_ref.forward(theta, T, scale)
    h2, _ = mlp_ref.forward(theta, -T, scale)
    assert np.allclose(h1, -h2, rtol=0, atol=1e-15)
