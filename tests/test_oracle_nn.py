"""Pins of the FP64 numpy U-Net used to check the warm-start kernels.

The periodic convolution against scipy.ndimage.correlate (mode "wrap"), the
pooling / upsampling adjoints by the dot-product test, and the whole
hand-written backward pass by central finite differences of the loss.
"""
import numpy as np
import pytest

from oracle import nn

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((6, 5, 7, 3))
    w = rng.standard_normal((2, 27, 3))
    b = rng.standard_normal(2)
    y = nn.conv(x, w, b)
    for co in range(2):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[co, :, ci].reshape(3, 3, 3)  # [dz+1, dy+1, dx+1]
            ref += scipy_ndimage.correlate(x[..., ci], k, mode="wrap")
        np.testing.assert_allclose(y[..., co], ref, atol=1e-12)


@pytest.mark.parametrize("taps", [27, 1])
def test_conv_backward_is_the_adjoint(taps):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 4, 3))
    w = rng.standard_normal((5, taps, 3))
    dz = rng.standard_normal((4, 6, 4, 5))
    dx, dw, db = nn.conv_bwd(x, w, dz)
    # <dz, conv(x)> is linear in x and w: its gradients are dx and dw
    f = lambda xx, ww: float((dz * nn.conv(xx, ww, np.zeros(5))).sum())  # noqa: E731
    e = 1e-6
    for _ in range(5):
        i = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[i] += e
        xm[i] -= e
        assert abs((f(xp, w) - f(xm, w)) / (2 * e) - dx[i]) < 1e-7
        j = tuple(rng.integers(0, s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[j] += e
        wm[j] -= e
        assert abs((f(x, wp) - f(x, wm)) / (2 * e) - dw[j]) < 1e-7
    np.testing.assert_allclose(db, dz.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 4, 3))
    d = rng.standard_normal((2, 2, 2, 3))
    assert abs((nn.pool(x) * d).sum() - (x * nn.pool_bwd(d)).sum()) < 1e-12
    lo = rng.standard_normal((2, 2, 2, 3))
    sk = rng.standard_normal((4, 4, 4, 2))
    du = rng.standard_normal((4, 4, 4, 5))
    dlo, dsk = nn.up_concat_bwd(du, 3)
    assert abs((nn.up_concat(lo, sk) * du).sum() - (lo * dlo).sum() - (sk * dsk).sum()) < 1e-12


def test_unet_backward_by_finite_differences():
    rng = np.random.default_rng(3)
    S = 8
    params = {n: [rng.standard_normal((co, t, ci)) * np.sqrt(2.0 / (ci * t)), rng.standard_normal(co) * 0.1]
              for n, ci, co, t, r, lvl in nn.LAYERS}
    x = rng.standard_normal((S, S, S, 16))
    base = rng.standard_normal((S, S, S, 5))
    target = rng.standard_normal((S, S, S, 5))
    fluid = (rng.uniform(size=(S, S, S)) > 0.2).astype(float)
    y, a = nn.forward(params, x)
    L, dy = nn.loss(y, base, target, fluid)
    g = nn.backward(params, a, dy)
    e = 1e-6
    for name in ("c0a", "c1b", "c2a", "c3", "c4", "head"):
        for k, idx in (("w", 0), ("b", 1)):
            arr = params[name][idx]
            j = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[j]
            arr[j] = old + e
            Lp = nn.loss(nn.forward(params, x)[0], base, target, fluid)[0]
            arr[j] = old - e
            Lm = nn.loss(nn.forward(params, x)[0], base, target, fluid)[0]
            arr[j] = old
            fd = (Lp - Lm) / (2 * e)
            an = g[f"{name}_{k}"][j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, k, fd, an)


def test_coarse_loss_pins():
    """The long-wavelength loss term: b = 1 is the masked MSE itself; an error
    field constant on each cube keeps its whole weight, one alternating in
    sign inside every cube has none; the gradient matches central finite
    differences of the loss."""
    rng = np.random.default_rng(5)
    S = 8
    y = rng.standard_normal((S, S, S, 16))
    base = rng.standard_normal((S, S, S, 5))
    target = rng.standard_normal((S, S, S, 5))
    fluid = (rng.uniform(size=(S, S, S)) > 0.25).astype(float)
    L1, g1 = nn.loss_coarse(y, base, target, fluid, 1)
    L0, g0 = nn.loss(y, base, target, fluid)
    assert abs(L1 - L0) <= 1e-13 * L0 and np.abs(g1 - g0).max() <= 1e-15
    # all fluid, error constant on each 4^3 cube: the cube means are the error itself
    ones = np.ones((S, S, S))
    e = np.repeat(np.repeat(np.repeat(rng.standard_normal((2, 2, 2, 5)), 4, 0), 4, 1), 4, 2)
    yc = np.zeros((S, S, S, 16))
    yc[..., :5] = e
    Lc, _ = nn.loss_coarse(yc, np.zeros((S, S, S, 5)), np.zeros((S, S, S, 5)), ones, 4)
    assert abs(Lc - (e[::4, ::4, ::4] ** 2).sum() / (S ** 3 * 5.0)) <= 1e-14
    # checkerboard error: every cube mean vanishes
    zz, yy, xx = np.meshgrid(np.arange(S), np.arange(S), np.arange(S), indexing="ij")
    yc[..., :5] = ((-1.0) ** (xx + yy + zz))[..., None] * np.arange(1, 6)
    assert nn.loss_coarse(yc, np.zeros((S, S, S, 5)), np.zeros((S, S, S, 5)), ones, 2)[0] < 1e-28
    L, g = nn.loss_coarse(y, base, target, fluid, 4)
    h = 1e-6
    for _ in range(12):
        j = tuple(int(rng.integers(0, s)) for s in (S, S, S)) + (int(rng.integers(0, 5)),)
        old = y[j]
        y[j] = old + h
        Lp = nn.loss_coarse(y, base, target, fluid, 4)[0]
        y[j] = old - h
        Lm = nn.loss_coarse(y, base, target, fluid, 4)[0]
        y[j] = old
        assert abs((Lp - Lm) / (2 * h) - g[j]) <= 1e-8 * max(1.0, abs(g[j]))
