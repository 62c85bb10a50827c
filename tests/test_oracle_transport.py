"""Pins for the oracle's transport: the CUI limiter's published branches,
constant density preserved by a discretely divergence-free flow, the
consistency identity C = U R for uniform velocity (Sec. 4.2.2's point:
mass and momentum fluxes share the same advective velocity and limited
density), and exact advection of a linear level set."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle import transport as tr
from oracle import levelset as ls
from oracle import operators as ops


def test_cui_branches():
    # linear monotone data: the kappa = 1/3 branch reproduces the midpoint
    assert tr.cui(0.0, 1.0, 2.0) == pytest.approx(1.5)
    # normalized branches
    f = lambda t: tr.cui(0.0, t, 1.0)
    assert f(0.1) == pytest.approx(0.3)                   # 3t
    assert f(0.5) == pytest.approx(5 * 0.5 / 6 + 1 / 3)  # 5t/6 + 1/3
    assert f(0.9) == pytest.approx(1.0)                   # 1
    assert f(1.5) == pytest.approx(1.5)                   # upwind outside [0,1]
    assert f(-0.2) == pytest.approx(-0.2)
    assert tr.cui(2.0, 2.0, 2.0) == 2.0                   # flat data
    # continuity of the piecewise map
    for t0 in (2 / 13, 0.8):
        assert f(t0 - 1e-12) == pytest.approx(f(t0 + 1e-12), abs=1e-9)


def _divfree_velocity(g, seed):
    """Discretely divergence-free MAC field: the discrete curl of a random
    edge potential, zero on walls."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((g.nz, g.ny + 1, g.nx + 1))  # z-potential on xy-edges
    A[:, 0, :] = A[:, -1, :] = 0.0
    A[:, :, 0] = A[:, :, -1] = 0.0
    u = (A[:, 1:, :] - A[:, :-1, :]) / g.hy
    v = -(A[:, :, 1:] - A[:, :, :-1]) / g.hx
    w = np.zeros(g.face_shape(2))
    return [u, v, w]


def test_constant_density_preserved_by_divfree_flow():
    g = Grid(9, 8, 6)
    vel = _divfree_velocity(g, 0)
    assert np.abs(ops.div(g, *vel)).max() < 1e-12
    rho = [np.full(g.face_shape(c), 3.7) for c in range(3)]
    R = tr.mass_flux(g, vel, rho)
    for c in range(3):
        assert np.abs(R[c]).max() < 1e-10


def test_consistency_uniform_velocity():
    """Where the velocity is uniform over the stencil, C = U R exactly."""
    g = Grid(14, 12, 10)
    U = np.array([0.3, -0.2, 0.1])
    rng = np.random.default_rng(1)
    vel = []
    for c in range(3):
        a = np.full(g.face_shape(c), U[c])
        # taper next to the walls so the field is a legal MAC velocity
        ax = 2 - c
        idx = [slice(None)] * 3
        for k in (0, 1, -2, -1):
            idx[ax] = k
            a[tuple(idx)] = 0.0
        vel.append(a)
    rho = [rng.uniform(1.0, 1000.0, g.face_shape(c)) for c in range(3)]
    R = tr.mass_flux(g, vel, rho)
    C = tr.convective(g, vel, rho)
    for c in range(3):
        inner = (slice(4, -4),) * 3
        assert np.allclose(C[c][inner], U[c] * R[c][inner], rtol=1e-12, atol=1e-9)


def test_linear_levelset_advected_exactly():
    g = Grid(12, 10, 8)
    phi = np.broadcast_to(g.cell_centers()[0] - 0.4, g.cell_shape).copy()
    Ux = 0.25
    vel = [np.full(g.face_shape(0), Ux) * g.interior_face_mask(0),
           np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    dt = 1e-2
    new = ls.advect(g, vel, phi, phi, dt)
    inner = new[:, :, 3:-3]
    assert np.allclose(inner, (phi - dt * Ux)[:, :, 3:-3], atol=1e-14)


# ---------------------------------------------------------------------------
# Time integration (Sec. 4.2.2): the extrapolated/interpolated stage
# velocities and the SSP-RK3 stages.

def test_rk_velocities_exact_for_polynomial_histories():
    """u^(1) approximates u^{n+1} and u^(2) approximates u^{n+1/2}
    (Sec. 4.2.2).  In the first cycle only u^n and u^{n-1} are known, and
    the two-point formulas are exact for velocities linear in time; later
    cycles also have u^{n+1,k}, and the three-point formula for u^(2) is
    exact for quadratics.  Each condition fixes every weight uniquely."""
    rng = np.random.default_rng(3)
    a, b, c = (rng.standard_normal((3, 4)) for _ in range(3))
    t, dt = 0.7, 0.13
    lin = lambda s: a + b * s
    quad = lambda s: a + b * s + c * s * s
    u1, u2 = tr.rk_velocities([lin(t)], [lin(t - dt)], None, 0)
    assert np.allclose(u1[0], lin(t + dt), rtol=0, atol=1e-14)
    assert np.allclose(u2[0], lin(t + 0.5 * dt), rtol=0, atol=1e-14)
    u1, u2 = tr.rk_velocities([quad(t)], [quad(t - dt)], [quad(t + dt)], 1)
    assert np.allclose(u1[0], quad(t + dt), rtol=0, atol=1e-14)
    assert np.allclose(u2[0], quad(t + 0.5 * dt), rtol=0, atol=1e-14)
    # a quadratic history defeats the first-cycle extrapolation (it is only
    # second-order accurate), which shows the test can fail
    u1, _ = tr.rk_velocities([quad(t)], [quad(t - dt)], None, 0)
    assert not np.allclose(u1[0], quad(t + dt), atol=1e-6)


def _x_uniform_velocity(g, U):
    """u = U on every x-face at least three faces from the x walls (tapered
    to zero on the wall faces), v = w = 0."""
    u = np.full(g.face_shape(0), U)
    u[:, :, 0] = u[:, :, -1] = 0.0
    u[:, :, 1] = u[:, :, -2] = U / 3.0
    u[:, :, 2] = u[:, :, -3] = 2.0 * U / 3.0
    return [u, np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]


def _face_x(g, c):
    return np.broadcast_to(g.face_centers(c)[0], g.face_shape(c))


def test_ssp_rk3_shifts_a_linear_density_by_the_integral_of_the_velocity():
    """A density linear in x carried by a uniform velocity U(t) moves by
    exactly -slope * integral of U over the step, and its momentum flux
    divergence is U(t^{n+1/2})^2 * slope.  The scheme's stage
    velocities (u^n, u^(1), u^(2)) and stage weights combine into Simpson's
    rule on [t^n, t^{n+1}] (exact for cubics), and the stage velocities
    themselves are exact for quadratic (later cycles) or linear (first
    cycle) histories, so the shift is exact to rounding.  Interior faces
    only (walls taper the flow)."""
    g = Grid(40, 5, 4, lx=2.0, ly=0.5, lz=0.4)
    s, t, dt = 0.8, 0.4, 0.05
    rho = [1.5 + s * _face_x(g, c) for c in range(3)]
    for k, U in ((1, lambda q: 0.6 + 0.5 * q - 0.9 * q * q), (0, lambda q: 0.6 + 0.5 * q)):
        un = _x_uniform_velocity(g, U(t))
        unm1 = _x_uniform_velocity(g, U(t - dt))
        uk = _x_uniform_velocity(g, U(t + dt))
        u1, u2 = tr.rk_velocities(un, unm1, uk, k)
        r3, C = tr.ssp_rk3(g, rho, un, u1, u2, dt)
        # integral of U over [t, t + dt], exact for the polynomial
        if k == 1:
            integ = 0.6 * dt + 0.25 * ((t + dt) ** 2 - t ** 2) - 0.3 * ((t + dt) ** 3 - t ** 3)
        else:
            integ = 0.6 * dt + 0.25 * ((t + dt) ** 2 - t ** 2)
        for c in range(3):
            inner = (slice(1, -1) if c == 2 else slice(None), slice(1, -1) if c == 1 else slice(None),
                     slice(12, -12))
            assert np.allclose(r3[c][inner], (rho[c] - s * integ)[inner], rtol=0, atol=1e-13), (k, c)
        # the convective term is built from the half-step velocity u^(2):
        # div(U rho U) = U^2 * slope for a uniform U and a linear rho
        inner = (slice(None), slice(None), slice(12, -12))
        assert np.allclose(C[0][inner], s * U(t + 0.5 * dt) ** 2, rtol=1e-12, atol=0), k


def _linear_regime_case():
    """A monotone density with a little curvature: every limiter evaluation
    in the interior falls in the kappa = 1/3 branch, where the limited face
    value is the linear combination (-q_U + 5 q_C + 2 q_D)/6, so the flux
    divergence R is a linear operator there."""
    g = Grid(48, 4, 4, lx=2.0, ly=0.4, lz=0.4)
    rho = [1.0 + 0.7 * _face_x(g, c) + 0.05 * _face_x(g, c) ** 2 for c in range(3)]
    return g, rho


def test_ssp_rk3_is_the_third_order_taylor_polynomial_on_a_linear_problem():
    """For a linear, time-independent right-hand side every three-stage
    third-order Runge-Kutta method advances y' = -R y by the Taylor
    polynomial y - dt R y + dt^2/2 R^2 y - dt^3/6 R^3 y; the SSP-RK3 weights
    (3/4, 1/4; 1/3, 2/3) are one such method.  The convective term uses the
    second stage (Sec. 4.2.2), an approximation to rho^{n+1/2}:
    rho^(2) = y - dt/2 R y + dt^2/4 R^2 y, and for a uniform velocity
    C = U R(rho^(2)) (the consistency identity).  R applications come from
    the oracle's flux divergence (pinned above)."""
    g, rho = _linear_regime_case()
    U, dt = 0.9, 0.02
    vel = _x_uniform_velocity(g, U)
    u1, u2 = tr.rk_velocities(vel, vel, None, 0)
    r3, C = tr.ssp_rk3(g, rho, vel, u1, u2, dt)
    R1 = tr.mass_flux(g, vel, rho)
    R2 = tr.mass_flux(g, vel, R1)
    R3 = tr.mass_flux(g, vel, R2)
    for c in range(3):
        inner = (slice(1, -1) if c == 2 else slice(None), slice(1, -1) if c == 1 else slice(None), slice(14, -14))
        taylor = rho[c] - dt * R1[c] + dt ** 2 / 2 * R2[c] - dt ** 3 / 6 * R3[c]
        assert np.allclose(r3[c][inner], taylor[inner], rtol=1e-14, atol=1e-14), c
        # the second-order and third-order terms are not negligible here
        assert np.abs((dt ** 2 / 2 * R2[c])[inner]).max() > 1e-5
        half = rho[c] - dt / 2 * R1[c] + dt ** 2 / 4 * R2[c]
        Rh = tr.mass_flux(g, vel, [half if d == c else rho[d] for d in range(3)])[c]
        if c == 0:
            assert np.allclose(C[0][inner], (U * Rh)[inner], rtol=1e-13, atol=1e-13)
        else:
            # no velocity along y or z: the transverse momenta are not convected
            assert np.abs(C[c][inner]).max() < 1e-13
    # the limiter really is in its linear branch over the compared region
    x = _face_x(g, 0)[0, 0]
    q = rho[0][0, 0]
    tt = (q[1:-1] - q[:-2]) / (q[2:] - q[:-2])
    assert np.all((tt[10:-10] > 2 / 13) & (tt[10:-10] <= 0.8))
