"""Pins for the oracle's IB4 transfers and rigid-body projection: the
kernel's defining moment conditions, discrete adjointness S_BC = J_BC^* at
walls (Sec. 3.3.2), exact reproduction of constant and linear fields, and
exact recovery of an imposed rigid motion (Sec. 4.2.5)."""
import numpy as np
import pytest

from oracle.grid import Grid, NO_SLIP, FREE_SLIP
from oracle import levelset
from oracle.ib import phi4, interpolate, spread
from oracle.rigid import rigid_fit, constrain, body_velocity
from paper_1901_07892_gb300 import inputs


def test_phi4_moment_conditions():
    rng = np.random.default_rng(0)
    for r in rng.uniform(0, 1, 200):
        j = np.arange(-3, 4)
        w = phi4(r - j)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)               # partition of unity
        assert ((r - j) * w).sum() == pytest.approx(0.0, abs=1e-14)   # first moment
        assert w[j % 2 == 0].sum() == pytest.approx(0.5, abs=1e-14)   # even/odd split
        assert (w * w).sum() == pytest.approx(3.0 / 8.0, abs=1e-14)  # sum of squares
    assert phi4(0.0) == pytest.approx(0.5)
    assert phi4(1.0) == pytest.approx(0.25)
    assert phi4(2.0) == 0.0 and phi4(2.5) == 0.0
    # continuity at |r| = 1
    assert phi4(1.0 - 1e-12) == pytest.approx(phi4(1.0 + 1e-12), abs=1e-9)


@pytest.mark.parametrize("bc", [(NO_SLIP,) * 6, (NO_SLIP, FREE_SLIP, NO_SLIP, FREE_SLIP, FREE_SLIP, NO_SLIP)])
def test_spread_is_adjoint_of_interp_at_walls(bc):
    g = Grid(9, 8, 7, lx=1.0, ly=0.9, lz=0.8, bc=bc)
    rng = np.random.default_rng(1)
    # markers everywhere, including within two cells of every wall
    X = np.stack([rng.uniform(0, g.lx, 300), rng.uniform(0, g.ly, 300), rng.uniform(0, g.lz, 300)], 1)
    F = rng.standard_normal((300, 3))
    vel = [rng.standard_normal(g.face_shape(c)) * g.interior_face_mask(c) for c in range(3)]
    dV = 1e-3
    SF = spread(g, F, X, dV)
    JU = interpolate(g, vel, X)
    lhs = sum((SF[c] * vel[c]).sum() for c in range(3)) * g.hx * g.hy * g.hz
    rhs = (F * JU).sum() * dV
    assert lhs == pytest.approx(rhs, rel=1e-13)
    for c in range(3):
        assert np.all(SF[c][~g.interior_face_mask(c)] == 0.0)


def test_interp_reproduces_linear_fields_inside():
    g = Grid(10, 10, 10)
    A = np.array([[0.1, 0.2, -0.3], [0.4, -0.5, 0.6], [-0.7, 0.8, 0.9]])
    c0 = np.array([1.0, -2.0, 0.5])
    vel = []
    for c in range(3):
        x, y, z = g.face_centers(c)
        val = c0[c] + A[c, 0] * x + A[c, 1] * y + A[c, 2] * z
        vel.append(np.broadcast_to(val, g.face_shape(c)).copy())
    rng = np.random.default_rng(2)
    X = rng.uniform(0.35, 0.65, (50, 3))
    U = interpolate(g, vel, X)
    ex = c0[None, :] + X @ A.T
    assert np.allclose(U, ex, atol=1e-13)


def test_rigid_fit_recovers_imposed_motion():
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (400, 3))
    Ur = np.array([0.3, -0.1, 0.2])
    Wr = np.array([0.05, 0.4, -0.3])
    Xc = X.mean(0)
    U = body_velocity(X, Xc, Ur, Wr)
    Ur2, Wr2, Xc2 = rigid_fit(X, U)
    assert np.allclose(Ur2, Ur, atol=1e-14)
    assert np.allclose(Wr2, Wr, atol=1e-13)


def test_projection_makes_body_rigid_inside():
    """Deep inside a half-cell marker lattice, S J is the identity on smooth
    fields, so after the correction J u equals the prescribed body velocity."""
    g = Grid(24, 24, 24)
    center, half = (0.5, 0.5, 0.5), (0.2, 0.2, 0.2)
    X, dV = inputs.marker_lattice(center, half, g.h)
    vel = [np.full(g.face_shape(c), 0.3 * (c + 1)) * g.interior_face_mask(c) for c in range(3)]
    new, Ub, Ur, Wr, Xc = constrain(g, vel, X, dV, [True] * 6, np.zeros(3), np.zeros(3))
    U = interpolate(g, new, X)
    deep = np.all(np.abs(X - 0.5) < 0.2 - 3 * g.hx, axis=1)
    assert deep.sum() > 100
    assert np.abs(U[deep]).max() < 1e-12
    # and the face velocities deep inside are zero
    for c in range(3):
        x, y, z = g.face_centers(c)
        m = (np.abs(x - 0.5) < 0.2 - 4 * g.hx) & (np.abs(y - 0.5) < 0.2 - 4 * g.hx) & (np.abs(z - 0.5) < 0.2 - 4 * g.hx)
        m = np.broadcast_to(m, g.face_shape(c))
        assert np.abs(new[c][m]).max() < 1e-12


def test_free_body_keeps_uniform_velocity():
    """A free body in a uniform flow takes the flow's velocity and leaves the
    field unchanged deep inside (momentum redistribution of a uniform field)."""
    g = Grid(20, 20, 20)
    X, dV = inputs.marker_lattice((0.5, 0.5, 0.5), (0.15, 0.15, 0.15), g.h)
    Uin = np.array([0.2, -0.1, 0.05])
    vel = [np.full(g.face_shape(c), Uin[c]) * g.interior_face_mask(c) for c in range(3)]
    new, Ub, Ur, Wr, Xc = constrain(g, vel, X, dV, [False] * 6, np.zeros(3), np.zeros(3))
    assert np.allclose(Ur, Uin, atol=1e-13)
    assert np.allclose(Wr, 0.0, atol=1e-12)
    for c in range(3):
        assert np.abs(new[c] - vel[c]).max() < 1e-13


def test_cylinder_sdf_closed_forms():
    """Signed distance to a capped cylinder along y (radius 0.2, half length
    0.3, centre (0.5, 0.5, 0.5)): on the axis at the centre -0.2 (the mantle
    is nearer than the caps); beside the mantle the radial gap; beyond a cap
    the axial gap; off a rim corner the Euclidean distance to the rim."""
    from oracle.grid import Grid
    g = Grid(10, 10, 10, 1.0, 1.0, 1.0, (-1.0,) * 6)
    c, R, hl = (0.5, 0.5, 0.5), 0.2, 0.3
    d = levelset.cylinder_sdf(g, c, R, hl)
    x, y, z = g.cell_centers()
    X, Y, Z = np.broadcast_arrays(x, y, z)

    def at(px, py, pz):
        k, j, i = int(pz * 10), int(py * 10), int(px * 10)
        return d[k, j, i], (X[k, j, i], Y[k, j, i], Z[k, j, i])

    v, (px, py, pz) = at(0.55, 0.55, 0.55)  # near the centre: inside, mantle nearest
    rr = np.hypot(px - 0.5, pz - 0.5)
    assert v == pytest.approx(max(rr - R, abs(py - 0.5) - hl))
    v, (px, py, pz) = at(0.95, 0.55, 0.55)  # beside the mantle
    assert v == pytest.approx(np.hypot(px - 0.5, pz - 0.5) - R)
    v, (px, py, pz) = at(0.55, 0.95, 0.55)  # beyond a cap
    assert v == pytest.approx(abs(py - 0.5) - hl)
    v, (px, py, pz) = at(0.95, 0.95, 0.95)  # off the rim
    assert v == pytest.approx(np.hypot(np.hypot(px - 0.5, pz - 0.5) - R, abs(py - 0.5) - hl))
    # a distance function: |grad d| = 1 away from the medial surfaces
    assert np.all(np.abs(d) <= np.sqrt(3.0))


def test_lm_force_closed_forms():
    """The Lagrange-multiplier force (Sec. 8): a body held at rest in a
    fluid moving uniformly at V inside it needs F = rho_s N dV V / dt to
    stop that fluid each step (U_b = 0, dU = -V on every marker); a free body,
    whose translation is the mean interpolated velocity, feels exactly its
    mass times its acceleration (the corrections dU sum to zero)."""
    from oracle.rigid import lm_force
    rng = np.random.default_rng(4)
    n, dV, dt, rho_s = 50, 1e-4, 2e-3, 700.0
    V = np.array([0.3, -0.2, 0.05])
    zero = np.zeros((n, 3))
    F = lm_force(zero, zero, np.tile(-V, (n, 1)), rho_s, dV, dt)
    assert np.allclose(F, rho_s * n * dV * V / dt, rtol=1e-14)
    X = rng.uniform(0.3, 0.7, (n, 3))
    Ui = rng.standard_normal((n, 3))
    Ur, Wr, Xc = rigid_fit(X, Ui)
    Ub = body_velocity(X, Xc, Ur, Wr)
    Ur_old = np.array([0.1, 0.0, -0.4])
    Ub_old = body_velocity(X, Xc, Ur_old, rng.standard_normal(3))
    F = lm_force(Ub, Ub_old, Ub - Ui, rho_s, dV, dt)
    assert np.allclose(F, rho_s * n * dV * (Ur - Ur_old) / dt, rtol=1e-10, atol=1e-10)


def test_lm_force_of_a_body_at_rest_in_a_tank_at_rest():
    """Hydrostatic three-phase tank with a locked box: u~ = 0 everywhere, so
    the body's Lagrange-multiplier force is zero."""
    from oracle import step as ost
    c = inputs.tank3d(n=10, with_body=True, dt=5e-4, gravity_mode="flow")
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                   gravity_mode="flow")
    s = ost.State(g, pr, c.phi, c.psi, ost.Body(c.markers, c.dV, [True] * 6, half=c.box_half))
    info = ost.step(s, c.dt)
    assert np.abs(info["F_lm"]).max() < 1e-6


def test_box_sdf_closed_forms():
    """The structure level set of a box (Sec. 4.1: the signed distance of
    the body about its centre): at hand-picked cell centres inside, beyond a
    face, beyond an edge and beyond a corner; and at every cell centre
    against the geometric definition (outside: the distance to the nearest
    point of the box, its clamp; inside: minus the distance to the nearest
    face)."""
    g = Grid(8, 8, 8)
    c = np.array([0.5, 0.5, 0.5])
    a = np.array([0.125, 0.25, 0.375])
    psi = levelset.box_sdf(g, c, a)
    # cell (i, j, k) is centred at ((i + 1/2)/8, ...); psi is indexed [k, j, i]
    assert psi[4, 4, 4] == pytest.approx(-0.0625, abs=1e-15)              # inside, nearest the x faces
    assert psi[4, 4, 7] == pytest.approx(0.3125, abs=1e-15)               # beyond the x+ face
    assert psi[4, 7, 7] == pytest.approx(np.hypot(0.3125, 0.1875), abs=1e-15)   # beyond the x+/y+ edge
    assert psi[7, 7, 7] == pytest.approx(np.sqrt(0.3125 ** 2 + 0.1875 ** 2 + 0.0625 ** 2), abs=1e-15)
    assert psi[0, 0, 0] == pytest.approx(np.sqrt(0.3125 ** 2 + 0.1875 ** 2 + 0.0625 ** 2), abs=1e-15)
    lo, hi = c - a, c + a
    x, y, z = np.broadcast_arrays(*g.cell_centers())
    p = np.stack([x, y, z], axis=-1)
    inside = np.all((p > lo) & (p < hi), axis=-1)
    outside_d = np.linalg.norm(p - np.clip(p, lo, hi), axis=-1)
    inside_d = np.minimum(p - lo, hi - p).min(axis=-1)
    ref = np.where(inside, -inside_d, outside_d)
    assert np.abs(psi - ref).max() < 1e-15
    assert inside.any() and (~inside).any()
