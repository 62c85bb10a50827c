"""Parity of the open top and the Dirichlet wave inlet (Sec. 7.1) with the
FP64 oracle: the operators with the open top's rows and ghosts (float64 and
double-float Stokes matvec, viscous, strain, pressure, gradient, divergence)
on ragged grids spanning several tiles, a strict Stokes solve whose pressure
is absolute (fixed by p = 0 on the top plane), and two steps of the wave
tank driven by the inlet through a tank with an open top, on both precision
paths, every velocity (the inlet faces included), the absolute pressure and
the level set compared."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.grid import Grid
from oracle.materials import Materials
from oracle import operators as ops
from oracle import step as ost
from oracle.solve import solve_stokes
from oracle.waves import StokesWave, Zones, Inlet
from paper_1901_07892_gb300 import inputs, wsi

OP_TOL = 1e-11
FIELD_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _grid(c):
    return Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc, open_top=c.open_top)


def _mat(c, g):
    return Materials(g, c.phi, c.psi, c.rho_l, c.rho_g, c.rho_s, c.mu_l, c.mu_g, c.mu_s, c.n_cells)


def _open_case(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    c = inputs.Case(nx=nx, ny=ny, nz=nz, lx=1.0, ly=0.9, lz=0.8)
    c.open_top = True
    x, y, z = c.cell_xyz()
    c.phi = np.broadcast_to(z - 0.45 * c.lz + 0.05 * np.sin(7 * x + 3 * y), (nz, ny, nx)).copy()
    c.psi = np.broadcast_to(inputs.box_distance((x, y, z), (0.5, 0.4, 0.35), (0.2, 0.15, 0.1)), (nz, ny, nx)).copy()
    return c, rng


@pytest.mark.parametrize("shape", [(37, 29, 11), (20, 9, 35), (31, 9, 17)])
def test_open_top_operator_parity(shape):
    c, rng = _open_case(*shape, 1)
    g = _grid(c)
    m = _mat(c, g)
    dt = 1e-3
    vel = [rng.standard_normal(g.face_shape(d)) * g.interior_face_mask(d) for d in range(3)]
    assert np.abs(vel[2][-1]).max() > 0  # the top faces are unknowns
    p = rng.standard_normal(g.cell_shape)
    x = g.pack(vel[0], vel[1], vel[2], p)
    ref = ops.stokes_apply(g, m, m.rho_face, dt, c.theta, x)
    for prec in (wsi.PREC_FP64, wsi.PREC_MIXED):
        ctx = wsi.Context.from_case(c, precision=prec)
        ctx.set_case(c)
        got = ctx.apply(wsi.OP_STOKES, torch.from_numpy(x).cuda(), dt).cpu().numpy()
        for a, b in zip(g.unpack(got), g.unpack(ref)):
            assert _rel(a, b) < OP_TOL, prec
        if prec == wsi.PREC_FP64:
            vflat = x[:ctx.nvel].copy()
            got = ctx.apply(wsi.OP_VISCOUS, vflat, dt)
            r = np.concatenate([a.ravel() for a in ops.viscous_apply(g, m, m.rho_face, dt, c.theta, *vel)])
            assert _rel(got, r) < OP_TOL
            got = ctx.apply(wsi.OP_STRAIN, vflat, dt)
            r = np.concatenate([a.ravel() for a in ops.strain_rate_apply(g, m, *vel)])
            assert _rel(got, r) < OP_TOL
            beta = [1.0 / a for a in m.rho_face]
            assert _rel(ctx.apply(wsi.OP_PRESSURE, p.ravel().copy(), dt),
                        ops.pressure_apply(g, beta, p).ravel()) < OP_TOL
            gr = np.concatenate([a.ravel() for a in ops.grad(g, p)])
            assert _rel(ctx.apply(wsi.OP_GRAD, p.ravel().copy(), dt), gr) < OP_TOL
            assert _rel(ctx.apply(wsi.OP_DIV, vflat, dt), ops.div(g, *vel).ravel()) < OP_TOL
        ctx.close()


@pytest.mark.parametrize("precision,smoother", [(wsi.PREC_FP64, wsi.SMOOTH_RBGS), (wsi.PREC_MIXED, wsi.SMOOTH_RBGS),
                                                (wsi.PREC_MIXED, wsi.SMOOTH_CHEBYSHEV)])
def test_open_top_solve_parity(precision, smoother):
    """A Stokes solve to rtol 1e-13 with gravity: the pressure is compared
    as it is (no mean removed), the open top fixes it; both multigrid
    smoothers carry the Dirichlet row of the top cells."""
    c, rng = _open_case(24, 12, 16, 2)
    g = _grid(c)
    m = _mat(c, g)
    dt = 1e-3
    bu = [rng.uniform(-1, 1, g.face_shape(d)) * 1e-2 * g.interior_face_mask(d) for d in range(3)]
    bu[2] = bu[2] + m.rho_face[2] * -9.81 * g.interior_face_mask(2)
    b = g.pack(bu[0], bu[1], bu[2], np.zeros(g.cell_shape))
    ref = g.unpack(solve_stokes(g, m, m.rho_face, dt, c.theta, b))
    ctx = wsi.Context.from_case(c, precision=precision, restart=40, mg_smoother=smoother)
    ctx.set_case(c)
    x, st = ctx.solve(torch.from_numpy(b).cuda(), dt, rtol=1e-13, max_iters=800)
    got = g.unpack(x.cpu().numpy())
    for a, r in zip(got, ref):
        assert _rel(a, r) < FIELD_TOL, (precision, st.iters)
    ctx.close()


def _inlet_tank(nx=32, ny=4, nz=16):
    c = inputs.wave_tank(nx=nx, ny=ny, nz=nz, with_bar=False)
    c.open_top = True
    w = c.extra["wave"]
    w["x_gen"] = 0.0
    return c


@pytest.mark.parametrize("precision,form", [(wsi.PREC_FP64, "consistent"), (wsi.PREC_MIXED, "consistent"),
                                            (wsi.PREC_FP64, "nonconservative")])
def test_inlet_open_top_step_parity(precision, form):
    """Two steps of a coarse wave tank (32 x 4 x 16 over 4 x 1 x 1, dt = 0.01)
    driven from rest by the inlet's second-order Stokes wave through an open
    top, damping zone at the far end; also with the non-conservative form,
    whose convection carries the inlet data of the half-step velocity."""
    c = _inlet_tank()
    g = _grid(c)
    w = c.extra["wave"]
    tf = wsi.FORM_CONSISTENT if form == "consistent" else wsi.FORM_NONCONSERVATIVE
    ctx = wsi.Context.from_case(c, precision=precision, restart=30, transport_form=tf)
    ctx.set_case(c, rho_s=c.rho_l, with_body=False)
    ctx.set_waves(w["H"], w["T"], w["depth"], 0.0, w["x_damp"], 0.0, 2, inlet=True)
    wave = StokesWave(w["H"], w["T"], w["depth"])
    pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                   gravity_mode="flow", n_cells=c.n_cells)
    s = ost.State(g, pr, c.phi, c.psi, None, zones=Zones(wave, 0.0, w["x_damp"], c.lx), inlet=Inlet(wave))
    for _ in range(2):
        ctx.step(c.dt, rtol=1e-13, max_iters=600)
        ost.step(s, c.dt, form=form)
    vel = ctx.get_field(wsi.F_VEL)
    o = np.cumsum([0] + [g.n_faces(d) for d in range(3)])
    vscale = max(np.abs(a).max() for a in s.vel)
    errs = {name: np.abs(vel[o[d]:o[d + 1]] - s.vel[d].ravel()).max() / vscale for d, name in enumerate("uvw")}
    errs["p"] = _rel(ctx.get_field(wsi.F_P), s.p.ravel())
    errs["phi"] = _rel(ctx.get_field(wsi.F_PHI), s.phi.ravel())
    print("inlet + open top, two steps, %s, %s form: per-field error against the oracle %s"
          % ("float64" if precision == wsi.PREC_FP64 else "mixed", form, {k: "%.2e" % v for k, v in errs.items()}))
    # the inlet faces hold the data of t^2 (the device's and numpy's
    # transcendental functions round differently)
    assert np.abs(s.vel[0][..., 0]).max() > 1e-3
    assert _rel(vel[o[0]:o[1]].reshape(g.face_shape(0))[..., 0], s.vel[0][..., 0]) < 1e-13
    # water leaves or enters through the top: the top faces move
    assert np.abs(s.vel[2][-1]).max() > 0
    for name in "uvw":
        assert errs[name] < FIELD_TOL, errs
    assert errs["p"] < FIELD_TOL, errs
    # the mixed path advects phi in float32 (the bound of the level-set parity tests)
    assert errs["phi"] < (1e-9 if precision == wsi.PREC_FP64 else 2e-6), errs
