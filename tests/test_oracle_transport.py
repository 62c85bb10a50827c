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
