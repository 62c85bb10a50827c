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
    return ou.bf16(a).astype(np.float32)


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
    """Against the float64 reference twice: with its storage rounded to
    bfloat16 where the kernels store bfloat16 (activations and the gradients
    passed between layers), which leaves only float32-vs-float64 accumulation
    and rare rounding-boundary flips (relative 1e-2 per layer); and without
    any rounding, where ten layers of bfloat16 storage give a few percent on
    the output."""
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
    x64 = np.transpose(x, (3, 0, 1, 2)).astype(np.float64)
    t64 = t[None].astype(np.float64)
    # no storage rounding in the reference: bfloat16 error budget
    ref, _ = ou.forward(P, x64)
    err = np.linalg.norm(out - ref[0]) / np.linalg.norm(ref[0])
    assert err < 3e-2, err
    # the kernels' storage decisions taken by the reference too
    ref, tape = ou.forward(P, x64, rnd=ou.bf16)
    err = np.linalg.norm(out - ref[0]) / np.linalg.norm(ref[0])
    assert err < 2e-3, err
    assert loss == pytest.approx(ou.loss(ref, t64), rel=2e-3)
    gr, _ = ou.backward(P, tape, ref, t64, rnd=ou.bf16)
    G = _pack_grads(gr, c0, c1, c2)
    off = 0
    shapes = ou.layer_shapes(3, c0, c1, c2)
    errs = {}
    for name in NAMES:
        co, ci = shapes[name]
        n = 27 * co * (16 if name == "a1" else ci) + co
        a, b = g[off:off + n], G[off:off + n]
        errs[name] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        off += n
    errs["head"] = float(np.linalg.norm(g[off:] - G[off:]) / np.linalg.norm(G[off:]))
    print("relative gradient error per layer", errs)
    assert max(errs.values()) < 1e-2, errs


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


def _train(net, level, mode, tanks, steps, rng, n):
    losses = []
    for tank_seed in tanks:
        c = _tank(tank_seed, n)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        wsi.attach_unet(ctx, net, level, enable=mode)
        for k in range(steps):
            lr = 2e-3 if len(losses) < 0.7 * steps * len(tanks) else 5e-4
            losses.append(wsi.unet_train_sample(ctx, _smooth_field(rng, n >> level), lr))
        ctx.close()
    return losses


def test_training_lowers_loss_and_gain_is_measured():
    """Train on exact pairs the solver's level operator generates (64^3 tanks,
    network on the 16^3 level) for each learned mode, then solve unseen
    tanks' pressure systems to 1e-8 with plain, replacing and augmenting
    cycles.  Every solve converges (the plain cycle judges each learned one
    and undoes it when it reduces the residual less, so a learned solve takes
    at most two cycles more than the plain one); the cycle counts and times
    are recorded."""
    n, level = 64, 2
    nc = n >> level
    nets, summary = {}, {"train": {}, "solves": []}
    for mode, flag in (("replace", wsi.LEARN_REPLACE), ("augment", wsi.LEARN_AUGMENT)):
        net = wsi.UNet(nc, nc, nc, 16, 32, 64, seed=11)
        t0 = time.time()
        losses = _train(net, level, flag, range(1000, 1006), 200, np.random.default_rng(5), n)
        summary["train"][mode] = {"steps": len(losses), "seconds": time.time() - t0,
                                  "loss_first50": float(np.mean(losses[:50])),
                                  "loss_last50": float(np.mean(losses[-50:]))}
        nets[mode] = (net, flag)
    for s in (2000, 2001, 2002):
        c = _tank(s, n)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        y = inputs.random_cells(c.phi.shape, s)
        y -= y.mean()
        row = {"seed": s}
        for mode in ("plain", "replace", "augment"):
            net, flag = nets.get(mode, (nets["replace"][0], wsi.LEARN_OFF))
            wsi.attach_unet(ctx, net, level, enable=flag)
            x, st = wsi.pressure_solve(ctx, y.ravel().copy(), rtol=1e-8, max_cycles=200)
            row[mode] = {"cycles": st.iters, "ms": st.ms, "rejected_at": st.learned_rejected,
                         "rel_residual": st.rel_residual}
        ctx.close()
        c64 = wsi.Context.from_case(c, precision=wsi.PREC_FP64)
        c64.set_case(c, with_body=False)
        x, st = wsi.pressure_solve(c64, y.ravel().copy(), rtol=1e-8, max_cycles=200)
        row["plain_fp64"] = {"cycles": st.iters, "ms": st.ms, "rel_residual": st.rel_residual}
        c64.close()
        summary["solves"].append(row)
    print(json.dumps(summary))
    for mode, tr in summary["train"].items():
        assert tr["loss_last50"] < 0.5 * tr["loss_first50"], (mode, tr)
    for row in summary["solves"]:
        for mode in ("plain", "replace", "augment", "plain_fp64"):
            assert row[mode]["rel_residual"] <= 1e-8, (mode, row)
        for mode in ("replace", "augment"):
            assert row[mode]["cycles"] <= row["plain"]["cycles"] + 2, row


def test_learned_guess_is_judged_against_the_zero_guess():
    """The initial-guess network trained on pairs the plain solver generates
    (right-hand side, solution) on 64^3 tanks, network on the 16^3 level:
    on unseen tanks every solve with the guess attached converges to 1e-8;
    the judge decides on every solve (kept or dropped); a dropped guess
    leaves exactly the plain solve (same cycles, same residual), a kept one
    costs at most two cycles more than plain."""
    n, level = 64, 2
    nc = n >> level
    net = wsi.UNet(nc, nc, nc, 16, 32, 64, seed=11)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    losses = []
    for tank_seed in (1000, 1001):
        c = _tank(tank_seed, n)
        plain = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        plain.set_case(c, with_body=False)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        wsi.attach_unet_guess(ctx, net, level)
        for _ in range(60):
            y = torch.rand(ctx.ncell, dtype=torch.float64, device="cuda", generator=gen) * 2.0 - 1.0
            y -= y.mean()
            x, st = wsi.pressure_solve(plain, y, rtol=1e-8, max_cycles=100)
            assert st.guess == -1
            losses.append(wsi.unet_train_guess(ctx, y, x, 1e-3))
        plain.close()
        ctx.close()
    assert all(np.isfinite(losses))
    rows = []
    for s in (2000, 2001):
        c = _tank(s, n)
        y = inputs.random_cells(c.phi.shape, s).ravel()
        y -= y.mean()
        plain = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        plain.set_case(c, with_body=False)
        _, sp = wsi.pressure_solve(plain, y.copy(), rtol=1e-8, max_cycles=200)
        ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
        ctx.set_case(c, with_body=False)
        wsi.attach_unet_guess(ctx, net, level)
        _, sg = wsi.pressure_solve(ctx, y.copy(), rtol=1e-8, max_cycles=200)
        rows.append((sp.iters, sp.rel_residual, sg.iters, sg.rel_residual, sg.guess))
        assert sg.rel_residual <= 1e-8 and sp.rel_residual <= 1e-8
        assert sg.guess in (0, 1)
        if sg.guess == 0:
            assert sg.iters == sp.iters and sg.rel_residual == sp.rel_residual
        else:
            assert sg.iters <= sp.iters + 2
        plain.close()
        ctx.close()
    print(json.dumps({"guess_loss_first10": float(np.mean(losses[:10])), "guess_loss_last10": float(np.mean(losses[-10:])),
                      "solves (plain its, res, guess its, res, kept)": rows}))
    net.close()
