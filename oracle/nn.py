"""FP64 numpy reference of the warm-start U-Net -- TEST INFRASTRUCTURE ONLY.

Plain NumPy in FP64: periodic 3x3x3 (or 1x1x1) convolutions written as sums
over taps of rolled arrays, ReLU, 2x2x2 mean pooling, nearest x2 upsampling
with channel concatenation, the masked mean-square error, and the hand-written
backward pass of each.  Arrays are channels last, shape (D, H, W, C); weights
(C_out, taps, C_in) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).  Only tests/ use
it; it shares no code with the CUDA kernels.
"""
from __future__ import annotations

import numpy as np

LAYERS = [("c0a", 16, 16, 27, 1, 0), ("c0b", 16, 16, 27, 1, 0), ("c1a", 16, 32, 27, 1, 1), ("c1b", 32, 32, 27, 1, 1),
          ("c2a", 32, 48, 27, 1, 2), ("c2b", 48, 48, 27, 1, 2), ("c3", 80, 32, 27, 1, 1), ("c4", 48, 16, 27, 1, 0),
          ("head", 16, 16, 1, 0, 0)]


def offsets(taps):
    if taps == 1:
        return [(0, 0, 0)]
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def shifted(x, off):
    """y[z,y,x] = x[z+dz, y+dy, x+dx] (periodic)."""
    dz, dy, dx = off
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def conv(x, w, b):
    out = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, off in enumerate(offsets(w.shape[1])):
        out += shifted(x, off) @ w[:, t, :].T
    return out + b


def conv_bwd(x, w, dz):
    """Gradients of sum(dz * conv(x, w, b)) w.r.t. x, w, b."""
    dw = np.zeros_like(w)
    dx = np.zeros_like(x)
    for t, off in enumerate(offsets(w.shape[1])):
        xs = shifted(x, off)
        dw[:, t, :] = np.einsum("zyxo,zyxi->oi", dz, xs)
        dx += np.roll(dz @ w[:, t, :], shift=off, axis=(0, 1, 2))
    return dx, dw, dz.sum(axis=(0, 1, 2))


def pool(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool_bwd(d):
    return np.repeat(np.repeat(np.repeat(d, 2, 0), 2, 1), 2, 2) / 8.0


def up_concat(lo, skip):
    up = np.repeat(np.repeat(np.repeat(lo, 2, 0), 2, 1), 2, 2)
    return np.concatenate([up, skip], axis=3)


def up_concat_bwd(d, c1):
    dlo = d[..., :c1]
    D, H, W, _ = dlo.shape
    dlo = dlo.reshape(D // 2, 2, H // 2, 2, W // 2, 2, c1).sum(axis=(1, 3, 5))
    return dlo, d[..., c1:]


def forward(params, x):
    """Returns (y, cache): y = head output (D, H, W, 16)."""
    a = {"x": x}
    r = lambda v: np.maximum(v, 0.0)  # noqa: E731
    a["c0a"] = r(conv(a["x"], *params["c0a"]))
    a["c0b"] = r(conv(a["c0a"], *params["c0b"]))
    a["p0"] = pool(a["c0b"])
    a["c1a"] = r(conv(a["p0"], *params["c1a"]))
    a["c1b"] = r(conv(a["c1a"], *params["c1b"]))
    a["p1"] = pool(a["c1b"])
    a["c2a"] = r(conv(a["p1"], *params["c2a"]))
    a["c2b"] = r(conv(a["c2a"], *params["c2b"]))
    a["u1"] = up_concat(a["c2b"], a["c1b"])
    a["c3"] = r(conv(a["u1"], *params["c3"]))
    a["u0"] = up_concat(a["c3"], a["c0b"])
    a["c4"] = r(conv(a["u0"], *params["c4"]))
    y = conv(a["c4"], *params["head"])
    return y, a


def loss(y, base, target, fluid):
    """Masked MSE of base + y[..., :5] against target over fluid positions."""
    d = (y[..., :5] + base - target) * fluid[..., None]
    n = fluid.sum() * 5.0
    L = float((d * d).sum() / n)
    dy = np.zeros_like(y)
    dy[..., :5] = 2.0 * d / n
    return L, dy


def loss_coarse(y, base, target, fluid, b):
    """Long-wavelength term: the masked error averaged over cubes of b^3
    positions, E = mean over the cube of (base + y[..., :5] - target) [fluid],
    L = sum over cubes and components of E^2 / n with n the MSE's count
    (5 x fluid positions); dL/dy[p] = 2 E(cube of p) / (b^3 n) at fluid
    positions.  Written with explicit loops over the cubes."""
    D, H, W = fluid.shape
    d = (y[..., :5] + base - target) * fluid[..., None]
    n = fluid.sum() * 5.0
    L = 0.0
    dy = np.zeros_like(y)
    for z0 in range(0, D, b):
        for y0 in range(0, H, b):
            for x0 in range(0, W, b):
                E = d[z0:z0 + b, y0:y0 + b, x0:x0 + b].sum(axis=(0, 1, 2)) / float(b ** 3)
                L += float((E * E).sum())
                dy[z0:z0 + b, y0:y0 + b, x0:x0 + b, :5] = (2.0 * E / (b ** 3 * n)) * fluid[z0:z0 + b, y0:y0 + b,
                                                                                          x0:x0 + b, None]
    return L / n, dy


def backward(params, a, dy):
    g = {}
    relu = lambda d, act: d * (act > 0)  # noqa: E731
    d_c4, g["head_w"], g["head_b"] = conv_bwd(a["c4"], params["head"][0], dy)
    dz = relu(d_c4, a["c4"])
    d_u0, g["c4_w"], g["c4_b"] = conv_bwd(a["u0"], params["c4"][0], dz)
    d_c3, d_c0b = up_concat_bwd(d_u0, 32)
    dz = relu(d_c3, a["c3"])
    d_u1, g["c3_w"], g["c3_b"] = conv_bwd(a["u1"], params["c3"][0], dz)
    d_c2b, d_c1b = up_concat_bwd(d_u1, 48)
    dz = relu(d_c2b, a["c2b"])
    d_c2a, g["c2b_w"], g["c2b_b"] = conv_bwd(a["c2a"], params["c2b"][0], dz)
    dz = relu(d_c2a, a["c2a"])
    d_p1, g["c2a_w"], g["c2a_b"] = conv_bwd(a["p1"], params["c2a"][0], dz)
    d_c1b = d_c1b + pool_bwd(d_p1)
    dz = relu(d_c1b, a["c1b"])
    d_c1a, g["c1b_w"], g["c1b_b"] = conv_bwd(a["c1a"], params["c1b"][0], dz)
    dz = relu(d_c1a, a["c1a"])
    d_p0, g["c1a_w"], g["c1a_b"] = conv_bwd(a["p0"], params["c1a"][0], dz)
    d_c0b = d_c0b + pool_bwd(d_p0)
    dz = relu(d_c0b, a["c0b"])
    d_c0a, g["c0b_w"], g["c0b_b"] = conv_bwd(a["c0a"], params["c0b"][0], dz)
    dz = relu(d_c0a, a["c0a"])
    _, g["c0a_w"], g["c0a_b"] = conv_bwd(a["x"], params["c0a"][0], dz)
    return g


def pack_input(solid, q, R, pitch, w):
    """(D, H, W, 16) input: [solid, Q(5), R/32, pitch/64, 20 w, 0 ...]; solid (D,H,W) -1 fluid; q (5, D, H, W)."""
    D, H, W = solid.shape
    x = np.zeros((D, H, W, 16))
    x[..., 0] = (solid >= 0).astype(float)
    x[..., 1:6] = np.moveaxis(q, 0, -1)
    x[..., 6] = R / 32.0
    x[..., 7] = pitch / 64.0
    x[..., 8] = 20.0 * w
    return x
