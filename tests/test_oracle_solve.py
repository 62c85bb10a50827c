"""Pins for the oracle's Stokes solve: a manufactured divergence-free
solution converging at second order, the well-balanced hydrostatic state of
Sec. 5 (zero velocity to round-off with rho^flow g, spurious currents with
the full rho g), and a brute-force dense solve on a tiny grid."""
import numpy as np
import pytest
import sympy as sy

from oracle.grid import Grid, NO_SLIP, FREE_SLIP
from oracle.materials import Materials, edge_harmonic, face_average, flow_only
from oracle import operators as ops
from oracle.solve import solve_stokes, stokes_matrix
from paper_1901_07892_gb300 import inputs

X, Y, Z = sy.symbols("x y z")


def _lam(expr):
    f = sy.lambdify((X, Y, Z), expr, "numpy")
    return lambda x, y, z: np.broadcast_to(f(x, y, z), np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z))).astype(float)


class _Mat:
    pass


def _stokes_ms_error(n, dim):
    pi = sy.pi
    # u = curl-like field of a stream function: divergence free, zero on walls,
    # odd about every wall in its tangential directions
    psi = sy.sin(pi * X) ** 2 * sy.sin(pi * Y) ** 2 * (sy.sin(pi * Z) if dim == 3 else 1)
    u = sy.diff(psi, Y)
    v = -sy.diff(psi, X)
    w = sy.Integer(0)
    p = sy.cos(pi * X) * sy.cos(pi * Y) * (sy.cos(pi * Z) if dim == 3 else 1)
    rho = 1 + sy.Rational(1, 2) * sy.sin(X + 2 * Y + Z)
    mu = sy.Rational(1, 10) * (1 + sy.Rational(1, 2) * sy.cos(pi * X) * sy.cos(pi * Y) * sy.cos(pi * Z))
    dt, theta = 0.05, 0.5
    xs = (X, Y, Z)
    vel = [u, v, w]
    rhs = []
    for c in range(3):
        L = sum(sy.diff(mu * (sy.diff(vel[c], xs[d]) + sy.diff(vel[d], xs[c])), xs[d]) for d in range(3))
        rhs.append(rho / dt * vel[c] - theta * L + sy.diff(p, xs[c]))
    if dim == 3:
        g = Grid(n, n, n)
    else:
        g = Grid(n, n, 1, lz=1.0 / n, bc=(NO_SLIP,) * 4 + (FREE_SLIP,) * 2)
    mat = _Mat()
    mat.mu_cc = _lam(mu)(*g.cell_centers())
    mat.mu_xy = edge_harmonic(g, mat.mu_cc, 0, 1)
    mat.mu_xz = edge_harmonic(g, mat.mu_cc, 0, 2)
    mat.mu_yz = edge_harmonic(g, mat.mu_cc, 1, 2)
    rho_face = [_lam(rho)(*g.face_centers(c)) for c in range(3)]
    b = [_lam(rhs[c])(*g.face_centers(c)) * g.interior_face_mask(c) for c in range(3)]
    x = solve_stokes(g, mat, rho_face, dt, theta, g.pack(b[0], b[1], b[2], np.zeros(g.cell_shape)))
    uh = g.unpack(x)
    err_u = max(np.abs(uh[c] - _lam(vel[c])(*g.face_centers(c)) * g.interior_face_mask(c)).max() for c in range(3))
    pe = _lam(p)(*g.cell_centers())
    pe = pe - pe.mean()
    err_p = np.abs(uh[3] - pe).max()
    return err_u, err_p


def test_stokes_manufactured_second_order_2d():
    e = [_stokes_ms_error(n, 2) for n in (16, 32, 64)]
    ru = [np.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    rp = [np.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    assert min(ru) > 1.8, (e, ru)
    assert min(rp) > 1.5, (e, rp)


def test_stokes_manufactured_3d():
    e1 = _stokes_ms_error(8, 3)
    e2 = _stokes_ms_error(16, 3)
    assert np.log2(e1[0] / e2[0]) > 1.7, (e1, e2)


def _tank2d_solve(n, mode):
    c = inputs.tank2d(n=n, with_body=True)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    rho_s = c.rho_l  # prescribed body: rho_s = max fluid density (Sec. 5)
    mat = Materials(g, c.phi, c.psi, c.rho_l, c.rho_g, rho_s, c.mu_l, c.mu_g, c.mu_s)
    if mode == "flow":
        rg = [flow_only(face_average(g, c.phi, d), c.rho_l, c.rho_g, mat.eps) for d in range(3)]
    else:
        rg = mat.rho_face
    b = [rg[d] * c.gravity[d] * g.interior_face_mask(d) for d in range(3)]
    x = solve_stokes(g, mat, mat.rho_face, c.dt, 0.5, g.pack(b[0], b[1], b[2], np.zeros(g.cell_shape)))
    return g, g.unpack(x), b


def test_hydrostatic_well_balanced_zero_velocity():
    """Sec. 5: with rho^flow g the discrete solution is u = 0 exactly (the
    force is a discrete gradient); the full rho g drives spurious flow."""
    g, (u, v, w, p), b = _tank2d_solve(32, "flow")
    umax = max(np.abs(u).max(), np.abs(v).max())
    assert umax < 1e-13
    # the pressure gradient balances the force exactly on interior faces
    G = ops.grad(g, p)
    assert np.abs(G[1] - b[1]).max() < 1e-9 * np.abs(b[1]).max()
    g, (u2, v2, w2, p2), _ = _tank2d_solve(32, "full")
    assert max(np.abs(u2).max(), np.abs(v2).max()) > 1e-6


def test_dense_bruteforce_tiny():
    g = Grid(4, 3, 3, lx=1.0, ly=0.8, lz=0.7)
    rng = np.random.default_rng(7)
    # moderate coefficients keep the system well conditioned, so two
    # different solvers must agree to near machine precision
    mat = Materials(g, rng.uniform(-0.3, 0.3, g.cell_shape), rng.uniform(-0.3, 0.3, g.cell_shape),
                    2.0, 1.0, 1.5, 0.2, 0.1, 0.2)
    dt = 0.1
    nt = sum(g.sizes())
    unk = g.unknown_mask()
    # dense matrix by applying to every unit vector (no colouring, no sparse)
    E = np.eye(nt)[unk]
    Kd = ops.stokes_apply(g, mat, mat.rho_face, dt, 0.5, E).T[unk]
    b = rng.standard_normal(nt) * unk
    u, v, w, p = g.unpack(b)
    b = g.pack(u, v, w, np.zeros_like(p))
    # minimum-norm least squares on the singular system, then zero-mean p
    sol = np.linalg.lstsq(Kd, b[unk], rcond=None)[0]
    xd = np.zeros(nt)
    xd[unk] = sol
    ud, vd, wd, pd = g.unpack(xd)
    pd -= pd.mean()
    xs = solve_stokes(g, mat, mat.rho_face, dt, 0.5, b)
    us = g.unpack(xs)
    for a, bb in zip((ud, vd, wd, pd), us):
        assert np.allclose(a, bb, rtol=1e-10, atol=1e-11 * np.abs(bb).max())
    # sparse assembly equals the dense probe
    Ks = stokes_matrix(g, mat, mat.rho_face, dt, 0.5).toarray()[unk][:, unk]
    assert np.allclose(Ks, Kd, rtol=1e-14, atol=1e-9)
