"""The learned pressure correction: the CUDA network's forward pass and
gradients against the float64 reference (tensor-core BF16 arithmetic: a few
percent), training on solver-generated pairs lowers the loss, and the gain of
the trained correction in a float64-residual pressure solve is measured
against plain multigrid on unseen tanks (the plain cycle stays the judge: a
failing learned cycle falls back)."""
import json
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet as ou
from paper_1901_07892_gb300 import inputs, wsi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = ["a1", "a2", "b1", "b2", "c1", "c2", "ub1", "ub2", "ua1", "ua2"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _bf16(a):
    """Round float32 values to bfloat16 (nearest-even) and back."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _unpack(p, c0, c1, c2):
    """GPU flat parameters -> oracle dictionary (a1's padded channels dropped)."""
    shapes = ou.layer_shapes(3, c0, c1, c2)
    d, off = {}, 0
    for name in NAMES:
        co, ci = shapes[name]
        cig = 16 if name == "a1" else ci
        n = 27 * co * cig
        w = p[off:off + n].reshape(27, co, cig)[:, :, :ci]
        d[name + ".w"] = np.transpose(w, (1, 2, 0)).reshape(co, ci, 3, 3, 3).astype(np.float64)
        off += n
        d[name + ".b"] = p[off:off + co].astype(np.float64)
        off += co
    d["head.w"] = p[off:off + c0].reshape(1, c0, 1, 1, 1).astype(np.float64)
    d["head.b"] = p[off + c0:off + c0 + 1].astype(np.float64)
    return d


def _pack_grads(g, c0, c1, c2):
    shapes = ou.layer_shapes(3, c0, c1, c2)
    out = []
    for name in NAMES:
        co, ci = shapes[name]
        cig = 16 if name == "a1" else ci
        w = np.transpose(g[name + ".w"].reshape(co, ci, 27), (2, 0, 1))
        wp = np.zeros((27, co, cig))
        wp[:, :, :ci] = w
        out += [wp.ravel(), g[name + ".b"]]
    out += [g["head.w"].ravel(), g["head.b"]]
    return np.concatenate(out)


def test_forward_and_gradients_match_reference():
    c0, c1, c2 = 16, 32, 64
    net = wsi.UNet(8, 8, 8, c0, c1, c2, seed=3)
    rng = np.random.default_rng(0)
    p = _bf16(net.params())  # the kernels use bf16 weights
    net.set_params(p)
    x = _bf16(rng.standard_normal((8, 8, 8, 3)).astype(np.float32))
    t = rng.standard_normal((8, 8, 8)).astype(np.float32)
    out = net.forward(x)
    loss = net.backward(t)
    g = net.grads()
    P = _unpack(p, c0, c1, c2)
    ref, tape = ou.forward(P, np.transpose(x, (3, 0, 1, 2)).astype(np.float64))
    ref_loss = ou.loss(ref, t[None].astype(np.float64))
    gr, _ = ou.backward(P, tape, ref, t[None].astype(np.float64))
    err = np.linalg.norm(out - ref[0]) / np.linalg.norm(ref[0])
    assert err < 3e-2, err
    assert loss == pytest.approx(ref_loss, rel=5e-2)
    G = _pack_grads(gr, c0, c1, c2)
    # per layer: weights and biases
    off = 0
    shapes = ou.layer_shapes(3, c0, c1, c2)
    for name in NAMES:
        co, ci = shapes[name]
        n = 27 * co * (16 if name == "a1" else ci) + co
        a, b = g[off:off + n], G[off:off + n]
        assert np.linalg.norm(a - b) <= 6e-2 * np.linalg.norm(b) + 1e-12, name
        off += n
    assert np.linalg.norm(g[off:] - G[off:]) <= 3e-2 * np.linalg.norm(G[off:])


def _smooth_field(rng, n, modes=6):
    z, y, x = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    e = np.zeros((n, n, n))
    for _ in range(modes):
        k = rng.integers(0, 4, size=3)
        e += rng.standard_normal() * np.cos(np.pi * k[0] * x / n) * np.cos(np.pi * k[1] * y / n) * \
            np.cos(np.pi * k[2] * z / n)
    e += 0.05 * rng.standard_normal(e.shape)
    return e - e.mean()


def _tank(seed, n=64):
    c = inputs.tank3d(n=n, seed=seed, with_body=False)
    return c


def test_training_lowers_loss_and_gain_is_measured():
    n, level = 64, 2
    nc = n // 4
    net = wsi.UNet(nc, nc, nc, 16, 32, 64, seed=11)
    rng = np.random.default_rng(5)
    losses = []
    t0 = time.time()
    for tank_seed in range(6):
        c = _tank(1000 + tank_seed, n)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        wsi.attach_unet(ctx, net, level, enable=False)
        for _ in range(60):
            losses.append(wsi.unet_train_sample(ctx, _smooth_field(rng, nc), 2e-3))
        ctx.close()
    train_s = time.time() - t0
    first, last = np.mean(losses[:20]), np.mean(losses[-20:])
    assert last < 0.5 * first, (first, last)
    # gain on unseen tanks: V-cycles and time to 1e-8 of a pressure solve
    results = []
    for s in (2000, 2001, 2002):
        c = _tank(s, n)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        y = inputs.random_cells(c.phi.shape, s)
        y -= y.mean()
        row = {"seed": s}
        for mode in ("plain", "learned"):
            wsi.attach_unet(ctx, net, level, enable=(mode == "learned"))
            x, st = wsi.pressure_solve(ctx, y.ravel().copy(), rtol=1e-8, max_cycles=200)
            assert st.rel_residual <= 1e-8, (mode, st.rel_residual)
            row[mode] = {"cycles": st.iters, "ms": st.ms}
        results.append(row)
        ctx.close()
    summary = {"train_steps": len(losses), "train_seconds": train_s, "loss_first20": first, "loss_last20": last,
               "solves": results}
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    with open(os.path.join(ROOT, "gpurun_out", "learned_gain.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))
