"""Pins for the oracle's materials and operators against facts that do not
come from the oracle itself: closed forms, textbook matrices built another
way, summation-by-parts identities and manufactured solutions whose exact
derivatives come from sympy."""
import numpy as np
import pytest
import scipy.sparse as sp
import sympy as sy

from oracle.grid import Grid, NO_SLIP, FREE_SLIP
from oracle.materials import heaviside, two_stage, edge_harmonic, Materials, face_average
from oracle import operators as ops


def test_heaviside_closed_forms():
    eps = 0.1
    assert heaviside(0.0, eps) == pytest.approx(0.5, abs=1e-15)
    assert heaviside(-eps, eps) == pytest.approx(0.0, abs=1e-15)
    assert heaviside(eps, eps) == pytest.approx(1.0, abs=1e-15)
    assert heaviside(-1.0, eps) == 0.0 and heaviside(1.0, eps) == 1.0
    # odd symmetry about 1/2 and monotonicity
    r = np.linspace(-2 * eps, 2 * eps, 401)
    H = heaviside(r, eps)
    assert np.allclose(H + heaviside(-r, eps), 1.0, atol=1e-15)
    assert np.all(np.diff(H) >= -1e-15)
    # value at eps/2: (1 + 1/2 + 1/pi)/2
    assert heaviside(eps / 2, eps) == pytest.approx(0.5 * (1.5 + 1.0 / np.pi), rel=1e-15)


def test_two_stage_limits():
    eps = 0.05
    # deep in liquid / gas / solid
    assert two_stage(-1.0, 1.0, 1000.0, 1.2, 500.0, eps) == 1000.0
    assert two_stage(1.0, 1.0, 1000.0, 1.2, 500.0, eps) == pytest.approx(1.2, rel=1e-12)
    assert two_stage(1.0, -1.0, 1000.0, 1.2, 500.0, eps) == 500.0
    assert two_stage(-1.0, -1.0, 1000.0, 1.2, 500.0, eps) == 500.0
    # on the liquid-gas interface, away from the solid: arithmetic mean
    assert two_stage(0.0, 1.0, 1000.0, 1.2, 500.0, eps) == pytest.approx(500.6)


def test_edge_harmonic_by_hand():
    g = Grid(2, 2, 1, bc=(NO_SLIP,) * 4 + (FREE_SLIP,) * 2)
    mu = np.array([[[1.0, 2.0], [4.0, 8.0]]])  # [k, j, i]
    exy = edge_harmonic(g, mu, 0, 1)
    assert exy.shape == (1, 3, 3)
    # interior edge (i=1, j=1): four cells 1, 2, 4, 8
    assert exy[0, 1, 1] == pytest.approx(4.0 / (1 + 0.5 + 0.25 + 0.125))
    # wall edge (i=0, j=1) on the x- wall: cells (0,0)=1 and (0,1)=4, mirrored
    assert exy[0, 1, 0] == pytest.approx(4.0 / (2 * (1.0 + 0.25)))
    # corner edge: only cell 1
    assert exy[0, 0, 0] == pytest.approx(1.0)


def test_face_average_by_hand():
    g = Grid(3, 1, 1)
    a = np.array([[[1.0, 3.0, 7.0]]])
    f = face_average(g, a, 0)
    assert np.allclose(f, [[[1.0, 2.0, 5.0, 7.0]]])


def _neumann_1d(n, h):
    main = -2.0 * np.ones(n)
    main[0] = main[-1] = -1.0
    return sp.diags([np.ones(n - 1), main, np.ones(n - 1)], [-1, 0, 1]) / h ** 2


@pytest.mark.parametrize("shape", [(5, 4, 3), (7, 6, 1)])
def test_pressure_constant_beta_is_kron_laplacian(shape):
    nx, ny, nz = shape
    g = Grid(nx, ny, nz, lx=1.0, ly=0.7, lz=0.4)
    beta = [np.full(g.face_shape(c), 1.0) for c in range(3)]
    Ix, Iy, Iz = (sp.identity(n) for n in (nx, ny, nz))
    Lx = _neumann_1d(nx, g.hx)
    Ly = _neumann_1d(ny, g.hy)
    Lz = _neumann_1d(nz, g.hz) if nz > 1 else sp.csr_matrix((1, 1))
    # x fastest: index = (k*ny + j)*nx + i  ->  kron(z, kron(y, x))
    L = sp.kron(Iz, sp.kron(Iy, Lx)) + sp.kron(Iz, sp.kron(Ly, Ix)) + sp.kron(Lz, sp.kron(Iy, Ix))
    p = np.random.default_rng(1).standard_normal(g.n_cells)
    ref = L @ p
    got = ops.pressure_apply(g, beta, p.reshape(g.cell_shape)).ravel()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-10 * np.abs(ref).max())


def test_summation_by_parts_grad_div():
    g = Grid(6, 5, 4, lx=1.0, ly=0.8, lz=0.6)
    rng = np.random.default_rng(2)
    p = rng.standard_normal(g.cell_shape)
    vel = []
    for c in range(3):
        a = rng.standard_normal(g.face_shape(c))
        a *= g.interior_face_mask(c)
        vel.append(a)
    G = ops.grad(g, p)
    lhs = sum((G[c] * vel[c]).sum() for c in range(3))
    rhs = -(p * ops.div(g, *vel)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _rand_mat(g, seed):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-0.3, 0.3, g.cell_shape)
    psi = rng.uniform(-0.3, 0.3, g.cell_shape)
    return Materials(g, phi, psi, 1000.0, 1.2, 500.0, 1e-3, 1.8e-5, 1e-3)


@pytest.mark.parametrize("bc", [(NO_SLIP,) * 6, (NO_SLIP,) * 4 + (FREE_SLIP,) * 2])
def test_viscous_operator_symmetric(bc):
    """L_mu is symmetric on the unknowns for any positive mu (strain-rate
    form with harmonic edge viscosity); a transposed index or a wrong ghost
    sign breaks this."""
    g = Grid(5, 4, 3, lx=1.0, ly=0.9, lz=0.7, bc=bc)
    mat = _rand_mat(g, 3)
    rng = np.random.default_rng(4)

    def rand_vel():
        out = []
        for c in range(3):
            a = rng.standard_normal(g.face_shape(c)) * g.interior_face_mask(c)
            out.append(a)
        return out
    a, b = rand_vel(), rand_vel()
    La = ops.strain_rate_apply(g, mat, *a)
    Lb = ops.strain_rate_apply(g, mat, *b)
    s1 = sum((La[c] * b[c]).sum() for c in range(3))
    s2 = sum((Lb[c] * a[c]).sum() for c in range(3))
    assert s1 == pytest.approx(s2, rel=1e-12)
    # negative semi-definite
    assert sum((La[c] * a[c]).sum() for c in range(3)) < 0


def test_strain_rate_of_rigid_rotation_vanishes_inside():
    """grad u + grad u^T = 0 for a rigid rotation: L_mu u = 0 at faces whose
    stencil stays off the walls, for any mu."""
    g = Grid(8, 8, 8)
    mat = _rand_mat(g, 5)
    W = np.array([0.3, -0.2, 0.5])
    vel = []
    for c in range(3):
        x, y, z = g.face_centers(c)
        X = np.broadcast_arrays(x, y, z)
        R = [X[0] - 0.5, X[1] - 0.5, X[2] - 0.5]
        # (W x R)_c
        cr = [W[1] * R[2] - W[2] * R[1], W[2] * R[0] - W[0] * R[2], W[0] * R[1] - W[1] * R[0]]
        vel.append(cr[c] * g.interior_face_mask(c))
    L = ops.strain_rate_apply(g, mat, *vel)
    for c in range(3):
        inner = L[c][2:-2, 2:-2, 2:-2]
        assert np.abs(inner).max() < 1e-12


# ---------------------------------------------------------------- manufactured
X, Y, Z = sy.symbols("x y z")


def _lam(expr):
    f = sy.lambdify((X, Y, Z), expr, "numpy")
    return lambda x, y, z: np.broadcast_to(f(x, y, z), np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z))).astype(float)


def _pressure_ms_error(n, dim):
    p = sy.cos(sy.pi * X) * sy.cos(2 * sy.pi * Y) * (sy.cos(sy.pi * Z) if dim == 3 else 1)
    beta = 1 / (1 + sy.Rational(1, 2) * sy.sin(X + 2 * Y + 3 * Z))
    f = sum(sy.diff(beta * sy.diff(p, v), v) for v in (X, Y, Z))
    g = Grid(n, n, n if dim == 3 else 1, lz=1.0 if dim == 3 else 1.0 / n,
             bc=(NO_SLIP,) * 4 + ((NO_SLIP,) * 2 if dim == 3 else (FREE_SLIP,) * 2))
    pf, bf, ff = _lam(p), _lam(beta), _lam(f)
    bet = [bf(*g.face_centers(c)) for c in range(3)]
    ph = pf(*g.cell_centers())
    fex = ff(*g.cell_centers())
    got = ops.pressure_apply(g, bet, ph)
    return np.abs(got - fex).max()


def test_pressure_manufactured_second_order_3d():
    e1 = _pressure_ms_error(8, 3)
    e2 = _pressure_ms_error(16, 3)
    e3 = _pressure_ms_error(32, 3)
    assert np.log2(e1 / e2) > 1.8 and np.log2(e2 / e3) > 1.9


def _viscous_ms(n, dim):
    pi = sy.pi
    if dim == 3:
        u = sy.sin(pi * X) * sy.sin(pi * Y) * sy.sin(pi * Z)
        v = sy.sin(2 * pi * X) * sy.sin(pi * Y) * sy.sin(2 * pi * Z)
        w = sy.sin(pi * X) * sy.sin(2 * pi * Y) * sy.sin(pi * Z)
        mu = 1 + sy.Rational(1, 2) * sy.cos(pi * X) * sy.cos(pi * Y) * sy.cos(pi * Z)
        g = Grid(n, n, n)
    else:
        u = sy.sin(pi * X) * sy.sin(pi * Y)
        v = sy.sin(2 * pi * X) * sy.sin(pi * Y)
        w = sy.Integer(0)
        mu = 1 + sy.Rational(1, 2) * sy.cos(pi * X) * sy.cos(pi * Y)
        g = Grid(n, n, 1, lz=1.0 / n, bc=(NO_SLIP,) * 4 + (FREE_SLIP,) * 2)
    vel = [u, v, w]
    xs = (X, Y, Z)
    L = []
    for c in range(3):
        e = 0
        for d in range(3):
            e += sy.diff(mu * (sy.diff(vel[c], xs[d]) + sy.diff(vel[d], xs[c])), xs[d])
        L.append(e)
    muf = _lam(mu)

    class M:
        pass
    mat = M()
    mat.mu_cc = muf(*g.cell_centers())
    mat.mu_xy = edge_harmonic(g, mat.mu_cc, 0, 1)
    mat.mu_xz = edge_harmonic(g, mat.mu_cc, 0, 2)
    mat.mu_yz = edge_harmonic(g, mat.mu_cc, 1, 2)
    vh = [_lam(vel[c])(*g.face_centers(c)) * g.interior_face_mask(c) for c in range(3)]
    got = ops.strain_rate_apply(g, mat, *vh)
    errs = []
    for c in range(3 if dim == 3 else 2):
        ex = _lam(L[c])(*g.face_centers(c)) * g.interior_face_mask(c)
        errs.append(np.abs(got[c] - ex).max())
    return max(errs)


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_manufactured_second_order(dim):
    ns = (16, 32, 64) if dim == 2 else (8, 16, 32)
    e = [_viscous_ms(n, dim) for n in ns]
    rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, (e, rates)
