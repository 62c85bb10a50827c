"""Pins for the float64 reference of the learned correction network:
central finite differences of the loss match the back-propagated gradients
(every layer, the skip connections, pooling and up-sampling), and the 3x3x3
convolution reduces to a known stencil for a hand-set kernel."""
import numpy as np
import pytest

from oracle import unet


def test_conv3_matches_hand_stencil():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7))
    w = np.zeros((1, 1, 3, 3, 3))
    # discrete 7-point Laplacian
    w[0, 0, 1, 1, 1] = -6.0
    for dz, dy, dx in ((0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)):
        w[0, 0, dz, dy, dx] = 1.0
    out = unet.conv3(x, w, np.array([0.5]))
    xp = np.pad(x[0], 1)
    ref = (xp[2:, 1:-1, 1:-1] + xp[:-2, 1:-1, 1:-1] + xp[1:-1, 2:, 1:-1] + xp[1:-1, :-2, 1:-1] +
           xp[1:-1, 1:-1, 2:] + xp[1:-1, 1:-1, :-2] - 6 * x[0]) + 0.5
    assert np.allclose(out[0], ref, atol=1e-13)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = unet.init_params(rng, cin=3, c0=4, c1=4, c2=8)
    x = rng.standard_normal((3, 8, 8, 8))
    target = rng.standard_normal((1, 8, 8, 8))
    out, t = unet.forward(p, x)
    g, dx = unet.backward(p, t, out, target)
    h = 1e-6
    for name in ("a1.w", "b2.w", "c1.w", "ub1.w", "ua1.w", "ua2.b", "head.w"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = unet.loss(unet.forward(p, x)[0], target)
            flat[idx] = old - h
            lm = unet.loss(unet.forward(p, x)[0], target)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert fd == pytest.approx(an, rel=1e-5, abs=1e-10), name
    # input gradient
    for idx in rng.choice(x.size, size=4, replace=False):
        xf = x.reshape(-1)
        old = xf[idx]
        xf[idx] = old + h
        lp = unet.loss(unet.forward(p, x)[0], target)
        xf[idx] = old - h
        lm = unet.loss(unet.forward(p, x)[0], target)
        xf[idx] = old
        assert (lp - lm) / (2 * h) == pytest.approx(dx.reshape(-1)[idx], rel=1e-5, abs=1e-10)
