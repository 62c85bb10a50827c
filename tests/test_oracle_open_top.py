"""Pins for the oracle's open top (Sec. 7.1: zero tangential velocity and
zero pressure on the tank's top boundary) against facts that do not come
from the operators themselves:

* the discrete energy identity of the strain-rate operator: for any velocity
  that vanishes on the walls, the volume-weighted sum of u . L u is minus the
  dissipation written as a sum of squares over cells and edges, each face,
  edge or cell weighted by the part of its control volume inside the box
  (1/2 on the top plane, 1/4 on edges where two boundary planes meet);
* the same weights make G and -D adjoint (summation by parts with the
  pressure ghost -p) and the viscous operator symmetric;
* a one-cell column with free-slip sides reduces w's operator to 2 mu w_zz
  with w = 0 at the bottom and dw/dz = 0 at the top, whose eigenvalues are
  (8 mu / h^2) sin^2((2m - 1) pi / (4 nz)), m = 1 .. nz;
* a resting liquid under gravity has p = rho g (lz - z) exactly: zero on the
  top plane, not up to a constant.
"""
import numpy as np
import pytest

from oracle.grid import Grid, NO_SLIP, FREE_SLIP
from oracle.materials import Materials
from oracle import operators as ops
from oracle.solve import solve_stokes


def _rand_mat(g, seed):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-0.3, 0.3, g.cell_shape)
    psi = rng.uniform(-0.3, 0.3, g.cell_shape)
    return Materials(g, phi, psi, 1000.0, 1.2, 500.0, 1e-3, 1.8e-5, 1e-3)


def _rand_vel(g, rng):
    return [rng.standard_normal(g.face_shape(c)) * g.interior_face_mask(c) for c in range(3)]


def _face_weights(g, c):
    """Part of each c-face's control volume inside the box: 1, or 1/2 on the
    open top."""
    w = np.ones(g.face_shape(c))
    if c == 2 and g.open_top:
        w[-1] = 0.5
    return w


def _edge_weights(g, c, d):
    """1/2 for each boundary plane an edge of the (c, d) plane lies on."""
    shape = list(g.cell_shape)
    shape[2 - c] += 1
    shape[2 - d] += 1
    w = np.ones(shape)
    for a in (c, d):
        idx = [slice(None)] * 3
        idx[2 - a] = 0
        w[tuple(idx)] *= 0.5
        idx[2 - a] = -1
        w[tuple(idx)] *= 0.5
    return w


def _pad_along(g, q, a):
    """q extended by one tangential ghost on both sides of axis a."""
    ax = q.ndim - 1 - a
    lo = np.take(q, [0], axis=ax) * g.sign(a, 0)
    hi = np.take(q, [-1], axis=ax) * g.sign(a, 1)
    return np.concatenate([lo, q, hi], axis=ax)


def _dissipation(g, mat, vel):
    """Sum over cells of 2 mu (du_c/dx_c)^2 plus, over edges, the weighted
    mu_e (du_c/dx_d + du_d/dx_c)^2, tangential ghosts across boundary planes."""
    h = g.h
    out = 0.0
    for c in range(3):
        q = vel[c]
        ax = q.ndim - 1 - c
        n = q.shape[ax]
        dq = (np.take(q, np.arange(1, n), axis=ax) - np.take(q, np.arange(0, n - 1), axis=ax)) / h[c]
        out += (2.0 * mat.mu_cc * dq * dq).sum()
    mu_edge = {(0, 1): mat.mu_xy, (0, 2): mat.mu_xz, (1, 2): mat.mu_yz}
    for (c, d), mu_e in mu_edge.items():
        def dd(q, a):
            qp = _pad_along(g, q, a)
            ax = qp.ndim - 1 - a
            n = qp.shape[ax]
            return (np.take(qp, np.arange(1, n), axis=ax) - np.take(qp, np.arange(0, n - 1), axis=ax)) / h[a]
        gam = dd(vel[c], d) + dd(vel[d], c)
        out += (_edge_weights(g, c, d) * mu_e * gam * gam).sum()
    return out


@pytest.mark.parametrize("open_top", [False, True])
def test_energy_identity(open_top):
    g = Grid(5, 4, 6, lx=1.0, ly=0.9, lz=1.1, open_top=open_top)
    mat = _rand_mat(g, 1)
    vel = _rand_vel(g, np.random.default_rng(2))
    L = ops.strain_rate_apply(g, mat, *vel)
    lhs = sum((_face_weights(g, c) * vel[c] * L[c]).sum() for c in range(3))
    assert lhs == pytest.approx(-_dissipation(g, mat, vel), rel=1e-12)
    if open_top:
        # the top faces take part: dropping them breaks the identity
        assert np.abs(vel[2][-1]).max() > 0 and np.abs(L[2][-1]).max() > 0


def test_open_top_grad_div_adjoint():
    g = Grid(6, 5, 4, lx=1.0, ly=0.8, lz=0.6, open_top=True)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(g.cell_shape)
    vel = _rand_vel(g, rng)
    G = ops.grad(g, p)
    lhs = sum((_face_weights(g, c) * G[c] * vel[c]).sum() for c in range(3))
    assert lhs == pytest.approx(-(p * ops.div(g, *vel)).sum(), rel=1e-12)
    # p = 0 on the plane: the top gradient sees the ghost -p
    assert np.allclose(G[2][-1], -2.0 * p[-1] / g.hz, rtol=1e-14)


def test_open_top_viscous_symmetric_weighted():
    g = Grid(4, 5, 3, lx=0.8, ly=1.0, lz=0.7, open_top=True)
    mat = _rand_mat(g, 5)
    rng = np.random.default_rng(6)
    a, b = _rand_vel(g, rng), _rand_vel(g, rng)
    La = ops.strain_rate_apply(g, mat, *a)
    Lb = ops.strain_rate_apply(g, mat, *b)
    s1 = sum((_face_weights(g, c) * La[c] * b[c]).sum() for c in range(3))
    s2 = sum((_face_weights(g, c) * Lb[c] * a[c]).sum() for c in range(3))
    assert s1 == pytest.approx(s2, rel=1e-12)


def test_open_top_column_eigenvalues():
    nz, lz, mu = 12, 1.3, 0.7
    g = Grid(1, 1, nz, lx=0.2, ly=0.3, lz=lz, bc=(FREE_SLIP,) * 4 + (NO_SLIP, NO_SLIP), open_top=True)
    ones = np.ones(g.cell_shape)
    mat = Materials(g, -ones, ones, 1.0, 1.0, 1.0, mu, mu, mu)
    cols = []
    for k in range(1, nz + 1):
        w = np.zeros(g.face_shape(2))
        w[k] = 1.0
        L = ops.strain_rate_apply(g, mat, np.zeros(g.face_shape(0)), np.zeros(g.face_shape(1)), w)
        assert np.abs(L[0]).max() == 0 and np.abs(L[1]).max() == 0
        cols.append(L[2][1:, 0, 0])
    A = -np.array(cols).T
    ev = np.sort(np.linalg.eigvals(A).real)
    m = np.arange(1, nz + 1)
    exact = np.sort(8.0 * mu / g.hz ** 2 * np.sin((2 * m - 1) * np.pi / (4 * nz)) ** 2)
    assert np.allclose(ev, exact, rtol=1e-12)


def test_open_top_hydrostatic_pressure_is_absolute():
    g = Grid(4, 3, 6, lx=0.5, ly=0.4, lz=0.9, open_top=True)
    rho, grav, dt = 998.0, -9.81, 1e-3
    ones = np.ones(g.cell_shape)
    mat = Materials(g, -ones, ones, rho, rho, rho, 1e-3, 1e-3, 1e-3)
    b_w = rho * grav * np.ones(g.face_shape(2)) * g.interior_face_mask(2)
    b = g.pack(np.zeros(g.face_shape(0)), np.zeros(g.face_shape(1)), b_w, np.zeros(g.cell_shape))
    x = solve_stokes(g, mat, mat.rho_face, dt, 0.5, b)
    u, v, w, p = g.unpack(x)
    _, _, z = g.cell_centers()
    assert max(np.abs(a).max() for a in (u, v, w)) < 1e-10
    assert np.allclose(p, rho * -grav * (g.lz - z) * np.ones(g.cell_shape), rtol=1e-10, atol=1e-9)


def test_open_top_needs_no_slip_lid():
    with pytest.raises(ValueError):
        Grid(4, 4, 4, bc=(NO_SLIP,) * 5 + (FREE_SLIP,), open_top=True)
    with pytest.raises(ValueError):
        Grid(4, 4, 1, open_top=True)


def test_open_top_transport_ghost_is_even():
    """Across the open top the transport mirrors w evenly (dw/dz = 0): for a
    flow leaving downward through the top cell, with w halving from the top
    face to the face below, the limiter's upwind point is the top face and its
    far point the mirror image of the face below, i.e. a local extremum, so
    the upper control-volume face of the last interior w-face carries the
    first-order upwind value w_top (an odd mirror would feed the limiter a
    monotone profile and give 0.917 w_below instead)."""
    from oracle import transport
    g = Grid(3, 3, 6, lx=0.6, ly=0.6, lz=1.2, open_top=True)
    nz = g.nz
    vel = [np.zeros(g.face_shape(c)) for c in range(3)]
    w_below, w_top = -0.8, -0.4
    vel[2][1:nz - 1] = -1.0
    vel[2][nz - 1] = w_below
    vel[2][nz] = w_top
    rho = [np.ones(g.face_shape(c)) for c in range(3)]
    C = transport.convective(g, vel, rho)
    # the z-flux divergence of the w-face below the top: upper CV face (top
    # cell) minus lower CV face (the cell below it), over hz; u = v = 0
    adv_hi = 0.5 * (w_below + w_top)
    adv_lo = 0.5 * (-1.0 + w_below)
    lo = adv_lo * transport.cui(w_top, w_below, -1.0)  # adv_lo < 0: upwind from above
    expected = (adv_hi * w_top - lo) / g.hz
    assert np.allclose(C[2][nz - 1], expected, rtol=1e-14)
