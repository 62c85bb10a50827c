"""Parity at the full sizes the bench runs, element by element against the
FP64 oracle, so that launch shapes that only occur on large grids are held
to the same bounds as the small cases:

* the mixed path's double-float Stokes matvec on the 256^3 bench tank
  (its launch covers 256 z-planes of 8 x 32 blocks of 32 x 8 threads);
* the SSP-RK3 transport and the level-set advection at 256^3, where the
  z-marching kernels take their full 32-plane chunks (smaller grids halve the
  chunk to keep the SMs busy);
* IB4 interpolation and spreading with config 2's ~68k box markers at 128^3.

Bounds as in the small parity tests: 1e-11 for float64 (and double-float)
arithmetic; the float32 transport and level-set bounds of the mixed path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.grid import Grid
from oracle.materials import Materials
from oracle import operators as ops
from oracle import transport as otr
from oracle import levelset as ols
from oracle import ib as oib
from paper_1901_07892_gb300 import inputs, wsi

OP_TOL = 1e-11


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
    return Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)


def _mat(c, g):
    return Materials(g, c.phi, c.psi, c.rho_l, c.rho_g, c.rho_s, c.mu_l, c.mu_g, c.mu_s, c.n_cells)


def _flat(v):
    return np.concatenate([a.ravel() for a in v])


@pytest.fixture(scope="module")
def tank256():
    c = inputs.tank3d(n=256, seed=7, dt=5e-4)
    g = _grid(c)
    return c, g, _mat(c, g)


def test_stokes_matvec_bench_tank_256(tank256):
    """k_stokes_df (mixed context) and k_stokes (float64 context) on the
    bench workload's coefficients, a random velocity with a large mean (the
    cancellation the double-float arithmetic must survive) and a random
    pressure."""
    c, g, m = tank256
    rng = np.random.default_rng(21)
    vel = [(rng.standard_normal(g.face_shape(d)) + 10.0) * g.interior_face_mask(d) for d in range(3)]
    p = rng.standard_normal(g.cell_shape)
    x = g.pack(vel[0], vel[1], vel[2], p)
    ref = g.unpack(ops.stokes_apply(g, m, m.rho_face, c.dt, c.theta, x))
    xt = torch.from_numpy(x).cuda()
    for prec in (wsi.PREC_MIXED, wsi.PREC_FP64):
        ctx = wsi.Context.from_case(c, precision=prec)
        ctx.set_case(c)
        got = g.unpack(ctx.apply(wsi.OP_STOKES, xt, c.dt).cpu().numpy())
        for a, b in zip(got, ref):
            assert _rel(a, b) < OP_TOL, prec
        ctx.close()


def test_transport_and_levelset_256(tank256):
    """Cycle k = 1 of the SSP-RK3 face-density transport with its convective
    term, and one level-set advection, on the 256^3 tank with seeded
    velocities; float64 path to 1e-11, float32 path to its bounds."""
    c, g, m = tank256
    rng = np.random.default_rng(22)
    mk = lambda: [rng.uniform(-1, 1, g.face_shape(d)) * 0.3 * g.interior_face_mask(d) for d in range(3)]
    un, unm1, uk = mk(), mk(), mk()
    dt = 2e-4
    u1, u2 = otr.rk_velocities(un, unm1, uk, 1)
    r3, Co = otr.ssp_rk3(g, m.rho_face, un, u1, u2, dt)
    r3, Co = _flat(r3), _flat(Co)
    phih = c.phi + 0.01 * rng.standard_normal(c.phi.shape)
    lso = ols.advect(g, uk, c.phi, phih, 1e-3).ravel()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for prec, rtol_rho, rtol_c, rtol_ls in ((wsi.PREC_FP64, OP_TOL, OP_TOL, OP_TOL),
                                            (wsi.PREC_MIXED, 1e-6, 1e-5, 1e-7)):
        ctx = wsi.Context.from_case(c, precision=prec)
        ctx.set_case(c)
        rho, C = ctx.transport(dev(_flat(un)), dev(_flat(unm1)), dev(_flat(uk)), 1, dt)
        assert _rel(rho.cpu().numpy(), r3) < rtol_rho, prec
        assert _rel(C.cpu().numpy(), Co) < rtol_c, prec
        got = ctx.advect_levelset(dev(_flat(uk)), dev(c.phi.ravel()), dev(phih.ravel()), 1e-3)
        assert _rel(got.cpu().numpy(), lso) < rtol_ls, prec
        ctx.close()


def test_ib_transfers_config2_markers():
    """Config 2 (128^3, box 0.2 x 0.2 x 0.1 at the surface, one marker per
    half cell: ~68k markers): interpolation of a random field and spreading
    of random forces."""
    c = inputs.tank3d(n=128, seed=None, dt=5e-4)
    g = _grid(c)
    assert len(c.markers) > 60000
    rng = np.random.default_rng(23)
    vel = [rng.standard_normal(g.face_shape(d)) * g.interior_face_mask(d) for d in range(3)]
    ctx = wsi.Context.from_case(c)
    ctx.set_case(c)
    X = np.ascontiguousarray(c.markers)
    U = ctx.interp(torch.from_numpy(_flat(vel)).cuda(), torch.from_numpy(X.ravel()).cuda())
    assert _rel(U.cpu().numpy().reshape(-1, 3), oib.interpolate(g, vel, X)) < OP_TOL
    F = rng.standard_normal(X.shape)
    S = ctx.spread(torch.from_numpy(F.ravel()).cuda(), torch.from_numpy(X.ravel()).cuda(), c.dV)
    assert _rel(S.cpu().numpy(), _flat(oib.spread(g, F, X, c.dV))) < 1e-12
    ctx.close()
