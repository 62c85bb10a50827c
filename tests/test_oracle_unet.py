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


def test_bf16_storage_rounding():
    # bfloat16 keeps 8 significant bits: the spacing above 1 is 2**-7
    u = 2.0 ** -7
    vals = np.array([1.0, 1 + u / 2, 1 + 1.5 * u, 1 + u / 2 + 2 ** -20, -(1 + 1.5 * u), 3.0, 0.0, 2.0 ** -130])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 3.0, 0.0, 2.0 ** -130])
    assert np.array_equal(unet.bf16(vals), want)
    # relative error bound 2**-8 on random values, idempotent
    x = np.random.default_rng(2).standard_normal(1000) * 1e3
    r = unet.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
    assert np.array_equal(unet.bf16(r), r)


def test_storage_rounding_hook_is_only_rounding():
    """With an identity hook the reference is unchanged; with bfloat16 storage
    the output moves by no more than the rounding budget of ten layers."""
    rng = np.random.default_rng(3)
    p = unet.init_params(rng, cin=3, c0=4, c1=4, c2=8)
    x = rng.standard_normal((3, 8, 8, 8))
    a, _ = unet.forward(p, x)
    b, _ = unet.forward(p, x, rnd=lambda v: v)
    c, _ = unet.forward(p, x, rnd=unet.bf16)
    assert np.array_equal(a, b)
    assert 0 < np.linalg.norm(c - a) / np.linalg.norm(a) < 3e-2
