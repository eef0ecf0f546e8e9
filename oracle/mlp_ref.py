"""FP64 CPU reference of the direction network for h (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the plain NumPy
forward and backward pass against which the GPU's BF16 training and
inference kernels are checked.  The network maps a unit direction T to the
27 components of h_vpq(T) (Sec. 2: dG_vp/dx_q = h_vpq(T) / R^2):

  s = +1 if T lies in the upper half-space (T_z > 0, ties broken by T_y, T_x),
      else -1;  x = s T                      (h is odd: h(-T) = -h(T))
  z1 = W1 x + b1,  a1 = silu(z1)             (128)
  z2 = W2 a1 + b2, a2 = silu(z2)             (128)
  z3 = W3 a2 + b3, a3 = silu(z3)             (128)
  o  = W4 a3 + b4                            (27, W4 padded to 32 rows)
  h  = s * scale * o

Loss on a batch: mean over samples and the 27 outputs of (o - s y / scale)^2.
Parameters are one flat vector in the order W1 [128x3], b1, W2 [128x128],
b2, W3 [128x128], b3, W4 [32x128], b4 [32] (37,664 numbers).
"""
from __future__ import annotations

import numpy as np

SIZES = [("W1", (128, 3)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
         ("W3", (128, 128)), ("b3", (128,)), ("W4", (32, 128)), ("b4", (32,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def half_space_sign(T):
    T = np.asarray(T)
    up = (T[:, 2] > 0) | ((T[:, 2] == 0) & ((T[:, 1] > 0) | ((T[:, 1] == 0) & (T[:, 0] >= 0))))
    return np.where(up, 1.0, -1.0)


def forward(theta, T, scale):
    """h [n, 27] and the cache of intermediate values."""
    p = unpack(theta)
    s = half_space_sign(T)
    x = T * s[:, None]
    z1 = x @ p["W1"].T + p["b1"]
    a1 = silu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = silu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = silu(z3)
    o = (a3 @ p["W4"].T + p["b4"])[:, :27]
    h = s[:, None] * np.asarray(scale)[None, :] * o
    return h, dict(s=s, x=x, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, o=o)


def loss_and_grad(theta, T, y, scale):
    """Mean-squared loss in normalised units and its gradient (manual backprop)."""
    p = unpack(theta)
    _, c = forward(theta, T, scale)
    n = T.shape[0]
    tgt = c["s"][:, None] * y / np.asarray(scale)[None, :]
    r = c["o"] - tgt
    loss = float(np.mean(r ** 2))
    go = np.zeros((n, 32))
    go[:, :27] = 2.0 * r / (n * 27)
    g = {}
    g["W4"] = go.T @ c["a3"]
    g["b4"] = go.sum(0)
    da3 = go @ p["W4"]
    g3 = da3 * dsilu(c["z3"])
    g["W3"] = g3.T @ c["a2"]
    g["b3"] = g3.sum(0)
    da2 = g3 @ p["W3"]
    g2 = da2 * dsilu(c["z2"])
    g["W2"] = g2.T @ c["a1"]
    g["b2"] = g2.sum(0)
    da1 = g2 @ p["W2"]
    g1 = da1 * dsilu(c["z1"])
    g["W1"] = g1.T @ c["x"]
    g["b1"] = g1.sum(0)
    return loss, pack(g)


def loss_only(theta, T, y, scale):
    _, c = forward(theta, T, scale)
    tgt = c["s"][:, None] * y / np.asarray(scale)[None, :]
    return float(np.mean((c["o"] - tgt) ** 2))
