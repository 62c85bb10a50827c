"""Pins for the oracle's Dirichlet wave inlet (Sec. 7.1) against facts that
do not come from its own lifting:

* a manufactured steady Stokes flow, divergence-free and zero on every wall
  but the inlet, whose inlet values are the data: the discrete solution
  converges to it at second order (a wrong sign, factor or index in the
  lifting of the normal or the tangential data leaves an O(1) error);
* with an open top the volume entering through the inlet leaves through the
  top, to round-off (continuity with the lifted data);
* a uniform inflow that carries the inlet's own tangential velocity has no
  convective flux divergence in the first column away from the other walls;
* the boundary Heaviside: full wave velocity deep in the water, none above
  the smeared surface, half on it.
"""
import numpy as np
import pytest
import sympy as sy

from oracle.grid import Grid, NO_SLIP, FREE_SLIP
from oracle.materials import Materials, heaviside, char_spacing
from oracle import transport, waves
from oracle.solve import solve_stokes_inlet


def _const_mat(g, rho=1.0, mu=1.0):
    ones = np.ones(g.cell_shape)
    return Materials(g, -ones, ones, rho, rho, rho, mu, mu, mu)


def _manufactured():
    X, Z = sy.symbols("x z")
    psi = (1 - X) ** 2 * Z ** 2 * (1 - Z) ** 2
    u = sy.diff(psi, Z)
    w = -sy.diff(psi, X)
    p = sy.cos(sy.pi * X) * sy.cos(sy.pi * Z)
    lap = lambda f: sy.diff(f, X, 2) + sy.diff(f, Z, 2)
    fu = u - lap(u) + sy.diff(p, X)  # rho/dt = 1, theta = mu = 1
    fw = w - lap(w) + sy.diff(p, Z)
    L = lambda f: sy.lambdify((X, Z), f, "numpy")
    return L(u), L(w), L(p), L(fu), L(fw)


def _solve_manufactured(n, mf):
    u_e, w_e, p_e, fu, fw = mf
    g = Grid(n, 2, n, lx=1.0, ly=2.0 / n, lz=1.0, bc=(NO_SLIP, NO_SLIP, FREE_SLIP, FREE_SLIP, NO_SLIP, NO_SLIP))
    mat = _const_mat(g)
    xu, _, zu = np.broadcast_arrays(*g.face_centers(0))
    xw, _, zw = np.broadcast_arrays(*g.face_centers(2))
    bu = fu(xu, zu) * g.interior_face_mask(0)
    bw = fw(xw, zw) * g.interior_face_mask(2)
    b = g.pack(bu, np.zeros(g.face_shape(1)), bw, np.zeros(g.cell_shape))
    u_in = u_e(0.0, zu[:, :, 0])
    w_in = w_e(0.0, np.arange(n + 1)[:, None] * g.hz * np.ones((1, g.ny)))
    x = solve_stokes_inlet(g, mat, mat.rho_face, 1.0, 1.0, b, u_in, w_in)
    u, v, w, p = g.unpack(x)
    assert np.abs(v).max() < 1e-12
    return np.abs(u - u_e(xu, zu)).max(), np.abs(w - w_e(xw, zw)).max()


def test_manufactured_inlet_flow_second_order():
    mf = _manufactured()
    # the first cells next to the inlet carry the O(h) truncation of the
    # ghost rule, so the rate approaches 2 from below (1.6-1.75 here); with
    # the tangential data at factor 1 instead of 2, or either datum left out
    # of the lifting, the error stays at 1e-2..1e-1 on every grid
    errs = [_solve_manufactured(n, mf) for n in (16, 32, 64)]
    for (eu0, ew0), (eu1, ew1) in zip(errs, errs[1:]):
        assert np.log2(eu0 / eu1) > 1.5, errs
        assert np.log2(ew0 / ew1) > 1.5, errs
    assert errs[-1][0] < 5e-4 and errs[-1][1] < 5e-4, errs


def test_inflow_leaves_through_open_top():
    g = Grid(7, 3, 6, lx=1.4, ly=0.6, lz=0.9, open_top=True)
    rng = np.random.default_rng(8)
    phi = rng.uniform(-0.3, 0.3, g.cell_shape)
    mat = Materials(g, phi, np.ones(g.cell_shape), 1000.0, 1.2, 1000.0, 1e-3, 1.8e-5, 1e-3)
    b = g.pack(*(rng.standard_normal(g.face_shape(c)) * g.interior_face_mask(c) for c in range(3)),
               np.zeros(g.cell_shape))
    u_in = rng.uniform(0.0, 1.0, (g.nz, g.ny))
    w_in = rng.standard_normal((g.nz + 1, g.ny))
    x = solve_stokes_inlet(g, mat, mat.rho_face, 1e-3, 0.5, b, u_in, w_in)
    u, v, w, p = g.unpack(x)
    assert np.array_equal(u[..., 0], u_in)
    inflow = u_in.sum() * g.hy * g.hz
    outflow = w[-1].sum() * g.hx * g.hy
    assert outflow == pytest.approx(inflow, rel=1e-10)


def test_uniform_inflow_carries_its_tangential_velocity():
    g = Grid(8, 3, 10, lx=1.0, ly=0.5, lz=1.0)
    U, W = 0.7, -0.4
    vel = [np.zeros(g.face_shape(c)) for c in range(3)]
    vel[0][...] = U
    vel[0][..., -1] = 0.0  # the far wall
    vel[2][1:-1] = W       # w vanishes on the z-walls
    rho = [np.ones(g.face_shape(c)) for c in range(3)]
    data = W * np.ones((g.nz + 1, g.ny))
    C = transport.convective(g, vel, rho, inlet_w=data)
    # first column, rows two or more faces from the z-walls: nothing changes
    assert np.abs(C[2][3:-3, :, 0]).max() < 1e-12
    # with the no-slip ghost instead the same column sees a jump
    C0 = transport.convective(g, vel, rho)
    assert np.abs(C0[2][3:-3, :, 0]).min() > 0.1


def test_boundary_heaviside_limits():
    g = Grid(16, 2, 40, lx=4.0, ly=0.2, lz=1.0)
    wave = waves.StokesWave(H=0.02, T=2.0, d=0.6)
    inl = waves.Inlet(wave)
    t = 0.37
    eps = 2.0 * char_spacing(g)
    zf = (np.arange(g.nz) + 0.5) * g.hz
    un = inl.normal(g, t, 2.0)[:, 0]
    uw, _ = wave.velocity(0.0, zf - wave.d, t)
    phib = zf - wave.d - wave.eta(0.0, t)
    deep, dry = phib < -eps, phib > eps
    assert deep.any() and dry.any()
    assert np.array_equal(un[deep], uw[deep])
    assert np.all(un[dry] == 0.0)
    mid = np.abs(phib) <= eps
    assert np.allclose(un[mid], (1.0 - heaviside(phib[mid], eps)) * uw[mid], rtol=1e-15)
    # on the surface itself the liquid fraction is one half
    assert 1.0 - heaviside(0.0, eps) == pytest.approx(0.5)
    ze = np.arange(g.nz + 1) * g.hz
    wt = inl.tangential(g, t, 2.0)[:, 0]
    _, vw = wave.velocity(0.0, ze - wave.d, t)
    pe = ze - wave.d - wave.eta(0.0, t)
    assert np.array_equal(wt[pe < -eps], vw[pe < -eps]) and np.all(wt[pe > eps] == 0.0)
