"""Parity of the wave-tank relaxation zones (Sec. 7.1) and of a full
wave-tank step with the locked trapezoidal bar on the bed (markers within two
cells of the bottom wall exercise the wall-folded spreading of Sec. 3.3.2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.grid import Grid
from oracle import step as ost
from oracle.waves import StokesWave, Zones
from paper_1901_07892_gb300 import inputs, wsi


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _ctx(c, **kw):
    ctx = wsi.Context.from_case(c, **kw)
    ctx.set_case(c, rho_s=c.rho_l, with_body=c.markers is not None)
    w = c.extra["wave"]
    ctx.set_waves(w["H"], w["T"], w["depth"], w["x_gen"], w["x_damp"], 0.0, 2)
    return ctx


def test_wave_relaxation_parity():
    c = inputs.wave_tank(nx=64, ny=8, nz=32, with_bar=False)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    ctx = _ctx(c)
    w = c.extra["wave"]
    zones = Zones(StokesWave(w["H"], w["T"], w["depth"]), w["x_gen"], w["x_damp"], c.lx)
    rng = np.random.default_rng(0)
    vel = [rng.uniform(-0.1, 0.1, g.face_shape(d)) * g.interior_face_mask(d) for d in range(3)]
    phi = c.phi + 0.01 * rng.standard_normal(c.phi.shape)
    flat = np.concatenate([a.ravel() for a in vel])
    for t in (0.0, 0.37, 1.9):
        v2, p2 = ctx.wave_relax(t, flat, phi.ravel().copy())
        vo, po = zones.relax(g, vel, phi, t, c.n_cells)
        assert _rel(v2, np.concatenate([a.ravel() for a in vo])) < 1e-12
        assert _rel(p2, po.ravel()) < 1e-13


@pytest.mark.parametrize("precision", [wsi.PREC_FP64, wsi.PREC_MIXED])
def test_wave_tank_step_parity_xsppm7(precision):
    """The wave-tank step with the level set advected by xsPPM7 (Sec. 4.2.1)
    instead of the CUI stand-in."""
    c = inputs.wave_tank(nx=32, ny=4, nz=16)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    ctx = _ctx(c, precision=precision, restart=30, ls_limiter=wsi.LIMIT_XSPPM7)
    w = c.extra["wave"]
    zones = Zones(StokesWave(w["H"], w["T"], w["depth"]), w["x_gen"], w["x_damp"], c.lx)
    pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                   gravity_mode="flow")
    s = ost.State(g, pr, c.phi, c.psi, ost.Body(c.markers, c.dV, [True] * 6), zones=zones)
    for _ in range(2):
        ctx.step(c.dt, rtol=1e-13, max_iters=600)
        ost.step(s, c.dt, limiter="xsppm7")
    vel = ctx.get_field(wsi.F_VEL)
    assert _rel(vel, np.concatenate([a.ravel() for a in s.vel])) < 1e-6
    p = ctx.get_field(wsi.F_P)
    assert _rel(p - p.mean(), (s.p - s.p.mean()).ravel()) < 1e-6
    assert _rel(ctx.get_field(wsi.F_PHI), s.phi.ravel()) < (1e-9 if precision == wsi.PREC_FP64 else 2e-6)


@pytest.mark.parametrize("precision", [wsi.PREC_FP64, wsi.PREC_MIXED])
def test_wave_tank_step_parity(precision):
    """Two steps of a coarse wave tank (32 x 4 x 16 over 4 x 1 x 1, dt = 0.01)
    with the bar on the bed: generation zone driving the flow from rest."""
    c = inputs.wave_tank(nx=32, ny=4, nz=16)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    ctx = _ctx(c, precision=precision, restart=30)
    w = c.extra["wave"]
    zones = Zones(StokesWave(w["H"], w["T"], w["depth"]), w["x_gen"], w["x_damp"], c.lx)
    pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                   gravity_mode="flow")
    body = ost.Body(c.markers, c.dV, [True] * 6)
    s = ost.State(g, pr, c.phi, c.psi, body, zones=zones)
    for _ in range(2):
        ctx.step(c.dt, rtol=1e-13, max_iters=600)
        ost.step(s, c.dt)
    vel = ctx.get_field(wsi.F_VEL)
    o = np.cumsum([0] + [g.n_faces(d) for d in range(3)])
    # each component against the scale of the whole velocity (the span-wise
    # component is zero up to rounding)
    vscale = max(np.abs(a).max() for a in s.vel)
    errs = {name: np.abs(vel[o[d]:o[d + 1]] - s.vel[d].ravel()).max() / vscale for d, name in enumerate("uvw")}
    p = ctx.get_field(wsi.F_P)
    errs["p"] = _rel(p - p.mean(), (s.p - s.p.mean()).ravel())
    errs["phi"] = _rel(ctx.get_field(wsi.F_PHI), s.phi.ravel())
    print("wave tank, two steps, %s: per-field error against the oracle %s"
          % ("float64" if precision == wsi.PREC_FP64 else "mixed", {k: "%.2e" % v for k, v in errs.items()}))
    for name in "uvw":
        assert errs[name] < 1e-6, errs
    assert errs["p"] < 1e-6, errs
    assert errs["phi"] < 1e-9, errs
