"""Checkpoint / restart of the time-stepping state and U-Net save / load:
stepping on from a restored state reproduces the uninterrupted run bit for
bit, with and without a body (the spreading sums fixed-point integers, so
its result does not depend on the order of the atomic additions).  A
reloaded network continues Adam with the same moments and step count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1901_07892_gb300 import inputs, wsi

FIELDS = (wsi.F_VEL, wsi.F_VEL_OLD, wsi.F_P, wsi.F_PHI, wsi.F_PSI)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _ctx(c, prec, body):
    ctx = wsi.Context.from_case(c, precision=prec)
    ctx.set_case(c, with_body=body)
    return ctx


@pytest.mark.parametrize("prec", [wsi.PREC_FP64, wsi.PREC_MIXED])
@pytest.mark.parametrize("body", [False, True])
def test_restart_continues_the_run(tmp_path, prec, body):
    c = inputs.tank3d(n=32, seed=3, with_body=True)
    a = _ctx(c, prec, body)
    for _ in range(4):
        a.step(c.dt, rtol=1e-10)
    b = _ctx(c, prec, body)
    for _ in range(2):
        b.step(c.dt, rtol=1e-10)
    path = tmp_path / "state.bin"
    b.checkpoint(path)
    b.close()
    d = _ctx(c, prec, body)
    d.restore(path)
    for _ in range(2):
        d.step(c.dt, rtol=1e-10)
    fields = FIELDS + ((wsi.F_MARKERS,) if body else ())
    for f in fields:
        x, y = a.get_field(f), d.get_field(f)
        assert np.array_equal(x, y), f
    a.close()
    d.close()


@pytest.mark.parametrize("prec", [wsi.PREC_FP64, wsi.PREC_MIXED])
def test_restart_with_inlet_and_open_top(tmp_path, prec):
    """A wave tank driven by the Dirichlet inlet through an open top: the
    checkpoint carries the inlet's tangential data of u^n and u^{n-1}, and
    the restored run goes on bit for bit."""
    c = inputs.wave_tank(nx=32, ny=4, nz=16, with_bar=False)
    c.open_top = True
    w = c.extra["wave"]

    def mk():
        ctx = wsi.Context.from_case(c, precision=prec, restart=30)
        ctx.set_case(c, rho_s=c.rho_l, with_body=False)
        ctx.set_waves(w["H"], w["T"], w["depth"], 0.0, w["x_damp"], 0.0, 2, inlet=True)
        return ctx
    a = mk()
    for _ in range(4):
        a.step(c.dt, rtol=1e-10)
    b = mk()
    for _ in range(2):
        b.step(c.dt, rtol=1e-10)
    path = tmp_path / "inlet.bin"
    b.checkpoint(path)
    b.close()
    d = mk()
    d.restore(path)
    for _ in range(2):
        d.step(c.dt, rtol=1e-10)
    for f in FIELDS:
        assert np.array_equal(a.get_field(f), d.get_field(f)), f
    a.close()
    d.close()


def test_spreading_is_deterministic():
    """The same forces spread twice (and from a second context) give the
    same bits, with many markers landing on the same faces."""
    c = inputs.tank3d(n=48, seed=None, with_body=True)
    rng = np.random.default_rng(4)
    X = np.ascontiguousarray(c.markers)
    F = rng.standard_normal(X.shape)
    outs = []
    for _ in range(2):
        ctx = _ctx(c, wsi.PREC_FP64, True)
        outs.append(ctx.spread(F.ravel(), X.ravel(), c.dV))
        outs.append(ctx.spread(F.ravel(), X.ravel(), c.dV))
        ctx.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.abs(outs[0]).max() > 0


def test_restore_rejects_other_grid(tmp_path):
    c = inputs.tank3d(n=16, seed=1, with_body=False)
    a = _ctx(c, wsi.PREC_FP64, False)
    path = tmp_path / "s.bin"
    a.checkpoint(path)
    c2 = inputs.tank3d(n=20, seed=1, with_body=False)
    b = _ctx(c2, wsi.PREC_FP64, False)
    with pytest.raises(wsi.WsiError):
        b.restore(path)
    with pytest.raises(wsi.WsiError):
        b.restore(tmp_path / "missing.bin")


def test_unet_save_load_continues_adam(tmp_path):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((8, 8, 8, 3)).astype(np.float32)
    t = rng.standard_normal((8, 8, 8)).astype(np.float32)
    a = wsi.UNet(8, 8, 8, seed=1)
    for _ in range(3):
        a.forward(x)
        a.backward(t)
        a.adam(1e-3)
    path = tmp_path / "net.bin"
    a.save(path)
    b = wsi.UNet(8, 8, 8, seed=2)
    b.load(path)
    assert np.array_equal(a.params(), b.params())
    for net in (a, b):
        net.forward(x)
        net.backward(t)
        net.adam(1e-3)
    # the weight gradients sum with float32 atomics: equal to their rounding
    pa, pb = a.params(), b.params()
    assert np.abs(pa - pb).max() <= 1e-5 * np.abs(pa).max()
    # weights load into a network of another grid size with the same widths
    big = wsi.UNet(16, 16, 16, seed=3)
    big.load(path)
    with pytest.raises(wsi.WsiError):
        wsi.UNet(8, 8, 8, c0=16, c1=16, c2=32, seed=0).load(path)
