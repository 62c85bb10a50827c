"""Pins for the oracle's xsPPM7 level-set advection (Sec. 4.2.1; the limiter
is read as the seventh-order upwind-biased interpolant limited to the
monotonicity-preserving, extremum-sensitive bounds of Suresh and Huynh):
exactness of the interpolant for cell averages of degree-6 polynomials
(which fixes all seven weights), the limiter inactive on smooth monotone
data, no new extremum at a jump, a smooth extremum kept rather than
clipped, exact translation of a linear level set, constant preservation and
conservation of the flux form."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle import levelset as ls


def _cell_averages(coef, centers, h):
    """Exact averages of the polynomial sum coef[k] x^k over [c - h/2, c + h/2]."""
    P = np.polynomial.polynomial.polyint(coef)
    val = lambda x: np.polynomial.polynomial.polyval(x, P)
    return (val(centers + h / 2) - val(centers - h / 2)) / h


def test_interp7_exact_for_degree_six_averages():
    rng = np.random.default_rng(0)
    for deg in range(7):
        coef = rng.standard_normal(deg + 1)
        h = 0.37
        centers = (np.arange(-3, 4)) * h   # cells -3..3; the face lies at +h/2
        q = _cell_averages(coef, centers, h)
        got = ls.interp7(*q)
        exact = np.polynomial.polynomial.polyval(h / 2, coef)
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-12), deg
    # degree 7 is not reproduced (so the test can fail)
    coef = np.zeros(8)
    coef[7] = 1.0
    q = _cell_averages(coef, np.arange(-3, 4) * 1.0, 1.0)
    assert abs(ls.interp7(*q) - 0.5 ** 7) > 1e-4


def test_limiter_inactive_on_smooth_monotone_data():
    h = 1e-2
    for x0 in np.linspace(0.1, 2.0, 13):
        q = _cell_averages_fn(np.exp, x0 + np.arange(-3, 4) * h, h)
        assert ls.xsppm7(*q) == ls.interp7(*q)


def _cell_averages_fn(f, centers, h, n=64):
    # Gauss-Legendre average, accurate to rounding for smooth f
    t, w = np.polynomial.legendre.leggauss(n)
    return np.array([np.sum(w * f(c + 0.5 * h * t)) / 2.0 for c in centers])


def test_no_new_extremum_at_a_jump():
    for qs in ([0, 0, 0, 0, 0, 1, 1], [0, 0, 0, 0, 1, 1, 1], [0, 0, 0, 1, 1, 1, 1], [1, 1, 1, 1, 1, 0, 0],
               [0, 0, 1, 1, 1, 1, 1]):
        q = [float(a) for a in qs]
        f = ls.xsppm7(*q)
        lo, hi = min(q[3], q[4]), max(q[3], q[4])
        assert lo - 1e-15 <= f <= hi + 1e-15, (qs, f)
    # the unlimited interpolant does overshoot there
    assert ls.interp7(0, 0, 0, 0, 0, 1, 1) < -0.05


def test_smooth_extremum_is_kept():
    """Cell averages of cos near its maximum: the face value at the crest
    is the exact point value, above every neighbouring average (a
    total-variation-diminishing limiter clips it to them)."""
    h = 2e-2
    centers = -h / 2 + np.arange(-3, 4) * h   # the face at x = 0 is the crest
    q = _cell_averages_fn(np.cos, centers, h)
    f = ls.xsppm7(*q)
    assert f == pytest.approx(1.0, abs=1e-12)
    assert f > q.max() + 1e-5


def test_linear_levelset_translated_exactly():
    g = Grid(20, 6, 5)
    phi = np.broadcast_to(g.cell_centers()[0] - 0.4, g.cell_shape).copy()
    Ux = 0.25
    vel = [np.full(g.face_shape(0), Ux) * g.interior_face_mask(0), np.zeros(g.face_shape(1)),
           np.zeros(g.face_shape(2))]
    dt = 1e-2
    new = ls.advect(g, vel, phi, phi, dt, limiter="xsppm7")
    assert np.allclose(new[:, :, 5:-5], (phi - dt * Ux)[:, :, 5:-5], atol=1e-14)


def test_constant_preserved_and_flux_form_conserves():
    g = Grid(12, 9, 7)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((g.nz, g.ny + 1, g.nx + 1))
    A[:, 0, :] = A[:, -1, :] = 0.0
    A[:, :, 0] = A[:, :, -1] = 0.0
    vel = [(A[:, 1:, :] - A[:, :-1, :]) / g.hy, -(A[:, :, 1:] - A[:, :, :-1]) / g.hx, np.zeros(g.face_shape(2))]
    c = np.full(g.cell_shape, 2.5)
    assert np.allclose(ls.advect(g, vel, c, c, 1e-3, limiter="xsppm7"), c, atol=1e-12)
    phi = rng.standard_normal(g.cell_shape)
    new = ls.advect(g, vel, phi, phi, 1e-3, limiter="xsppm7")
    assert abs(new.sum() - phi.sum()) < 1e-10 * np.abs(phi).sum()


def test_mirror_symmetry_of_the_upwind_stencils():
    """Flow in -x sees the mirror image of the stencil of flow in +x: the
    update of a field mirrored in x with the mirrored velocity is the mirror
    of the update; and a linear level set moves exactly either way."""
    g = Grid(16, 5, 4)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal(g.cell_shape)
    u = rng.standard_normal(g.face_shape(0)) * g.interior_face_mask(0)
    vel = [u, np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    new = ls.advect(g, vel, phi, phi, 1e-2, limiter="xsppm7")
    velm = [-u[:, :, ::-1], np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    newm = ls.advect(g, velm, phi[:, :, ::-1].copy(), phi[:, :, ::-1].copy(), 1e-2, limiter="xsppm7")
    assert np.allclose(newm[:, :, ::-1], new, rtol=0, atol=1e-13)
    lin = np.broadcast_to(g.cell_centers()[0] - 0.4, g.cell_shape).copy()
    velx = [np.full(g.face_shape(0), -0.3) * g.interior_face_mask(0), np.zeros(g.face_shape(1)),
            np.zeros(g.face_shape(2))]
    moved = ls.advect(g, velx, lin, lin, 1e-2, limiter="xsppm7")
    assert np.allclose(moved[:, :, 5:-5], (lin + 1e-2 * 0.3)[:, :, 5:-5], atol=1e-14)
