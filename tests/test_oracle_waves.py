"""Pins for the oracle's Stokes-wave and relaxation-zone formulas (Sec. 7.1):
the paper's Case A parameters satisfy the dispersion relation (golden values
printed in Sec. 7.2), the textbook deep/shallow-water limits, the linear
kinematic surface condition, and the potential-flow identities of the
velocity field (divergence- and curl-free)."""
import json
import os

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.waves import StokesWave, wavenumber, alpha, Zones

GOLD = os.path.join(os.path.dirname(__file__), "golden", "stokes_wave_case_a.json")


def test_case_a_parameters_satisfy_dispersion():
    gd = json.load(open(GOLD))
    d, g = gd["d"], gd["g"]
    T = gd["T_over_sqrt_d_over_g"] * np.sqrt(d / g)
    k = wavenumber(2 * np.pi / T, d, g)
    lam = 2 * np.pi / k
    # the paper prints lambda/d to four significant digits
    assert lam / d == pytest.approx(gd["lambda_over_d"], rel=5e-4)


def test_dispersion_limits():
    g = 9.81
    # deep water: omega^2 = g k
    k = wavenumber(2.0, 100.0, g)
    assert k == pytest.approx(4.0 / g, rel=1e-12)
    # shallow water: omega = k sqrt(g d)
    d = 1e-4
    k = wavenumber(1e-3, d, g)
    assert 1e-3 / k == pytest.approx(np.sqrt(g * d), rel=1e-6)


def test_linear_kinematic_surface_condition():
    """d eta_1/dt = v_1 at y = 0 for the first-order parts, which holds only
    with the dispersion relation and the printed amplitude."""
    w = StokesWave(H=1e-10, T=1.3, d=0.7)   # tiny H: second order negligible
    x = np.linspace(0, w.lam, 17)
    t, dt = 0.3, 1e-7
    deta = (w.eta(x, t + dt) - w.eta(x, t - dt)) / (2 * dt)
    u, v = w.velocity(x, 0.0, t)
    assert np.allclose(deta, v, rtol=1e-6, atol=1e-22)


def test_velocity_is_potential_flow():
    w = StokesWave(H=0.05, T=1.0, d=0.5)
    x = np.linspace(0.1, 1.3, 11)[:, None]
    y = np.linspace(-0.45, 0.0, 9)[None, :]
    e = 1e-5
    ux = (w.velocity(x + e, y, 0.2)[0] - w.velocity(x - e, y, 0.2)[0]) / (2 * e)
    vy = (w.velocity(x, y + e, 0.2)[1] - w.velocity(x, y - e, 0.2)[1]) / (2 * e)
    uy = (w.velocity(x, y + e, 0.2)[0] - w.velocity(x, y - e, 0.2)[0]) / (2 * e)
    vx = (w.velocity(x + e, y, 0.2)[1] - w.velocity(x - e, y, 0.2)[1]) / (2 * e)
    scale = np.abs(w.velocity(x, y, 0.2)[0]).max() * w.k
    assert np.abs(ux + vy).max() < 1e-7 * scale
    assert np.abs(uy - vx).max() < 1e-7 * scale
    # bottom boundary: no normal velocity at y = -d
    assert np.abs(w.velocity(x, -0.5, 0.2)[1]).max() < 1e-15


def test_eta_second_order_amplitude():
    w = StokesWave(H=0.05, T=1.0, d=0.5)
    # crest minus trough exceeds H by the second-order term's contribution: 0
    # (cos 2th is +1 at both crest and trough); the mean level is zero
    x = np.linspace(0, w.lam, 4097)[:-1]
    e = w.eta(x, 0.0)
    assert e.max() - e.min() == pytest.approx(w.H, rel=1e-12)
    assert abs(e.mean()) < 1e-15


def test_alpha_profile():
    assert alpha(0.0) == pytest.approx(1.0)
    assert alpha(1.0) == pytest.approx(0.0, abs=1e-15)
    xb = np.linspace(0, 1, 101)
    assert np.all(np.diff(alpha(xb)) <= 0)


def test_relaxation_leaves_the_middle_untouched():
    g = Grid(32, 4, 8, lx=4.0, ly=0.5, lz=1.0)
    z = Zones(StokesWave(0.05, 1.0, 0.5), 0.5, 3.5, 4.0)
    rng = np.random.default_rng(0)
    vel = [rng.standard_normal(g.face_shape(c)) * g.interior_face_mask(c) for c in range(3)]
    phi = rng.standard_normal(g.cell_shape)
    new, phin = z.relax(g, vel, phi, 0.37)
    xc = g.cell_centers()[0]
    mid = np.broadcast_to((xc > 0.5) & (xc < 3.5), g.cell_shape)
    assert np.array_equal(phin[mid], phi[mid])
    # at the far walls the relaxed level set equals its target
    assert np.all(np.abs(new[0][:, :, -1]) == 0.0)


def _eta2_coefficient(w):
    """Amplitude of the cos(2 theta) term of eta: half the sum of eta at a
    crest phase (theta = 0) and a trough phase (theta = pi), where the
    first-order terms cancel."""
    return 0.5 * (w.eta(0.0, 0.0) + w.eta(0.5 * w.lam, 0.0))


def test_eta_second_order_deep_and_shallow_limits():
    """Textbook limits of the second-order Stokes surface (Sec. 7.1):
    deep water (kd >> 1): eta_2 = k H^2 / 8 (with a = H/2: k a^2 / 2);
    shallow water (kd << 1): eta_2 = 3 H^2 / (16 k^2 d^3)."""
    H = 0.01
    w = StokesWave(H=H, T=0.8, d=5.0)  # kd = 31: exp(-2kd) corrections are below rounding
    assert _eta2_coefficient(w) == pytest.approx(w.k * H * H / 8.0, rel=1e-10)
    w = StokesWave(H=1e-4, T=60.0, d=0.5)
    kd = w.k * w.d
    assert kd < 0.05
    # next term of the expansion is O((kd)^2) relative
    assert _eta2_coefficient(w) == pytest.approx(3.0 * w.H ** 2 / (16.0 * w.k ** 2 * w.d ** 3), rel=3 * kd ** 2)


def _kinematic_residual(w):
    """max |v - eta_t - u eta_x| on the actual free surface y = eta(x, t):
    the exact kinematic condition, with central differences of eta."""
    x = np.linspace(0.0, w.lam, 257)[:-1]
    t, e = 0.3, 1e-6
    eta = w.eta(x, t)
    eta_t = (w.eta(x, t + e) - w.eta(x, t - e)) / (2 * e)
    eta_x = (w.eta(x + e, t) - w.eta(x - e, t)) / (2 * e)
    u, v = w.velocity(x, eta, t)
    return np.abs(v - eta_t - u * eta_x).max()


def test_kinematic_surface_condition_holds_to_second_order():
    """A second-order Stokes wave satisfies the kinematic free-surface
    condition on its own surface up to O(H^3): halving H divides the residual
    by 8.  A wrong second-order coefficient of eta or of the vertical
    velocity (or a wrong sign of either) leaves an O(H^2) residual, which
    halving H divides by only 4."""
    r = [_kinematic_residual(StokesWave(H=H, T=1.0, d=0.5)) for H in (2e-3, 1e-3)]
    assert r[0] / r[1] > 7.0, r
    r = [_kinematic_residual(StokesWave(H=H, T=1.4, d=0.3)) for H in (2e-3, 1e-3)]
    assert r[0] / r[1] > 7.0, r


def test_second_order_velocity_is_curl_free_at_order_two():
    """The second-order parts of u_w and v_w derive from one potential
    (cosh/sinh of 2k(d+y) with cos/sin 2 theta), so they must carry the same
    coefficient: the curl of the velocity vanishes with the O(H^2) parts
    isolated (velocity at H minus twice the velocity at H/2 removes the
    first-order part exactly)."""
    x = np.linspace(0.1, 1.3, 11)[:, None]
    y = np.linspace(-0.45, 0.0, 9)[None, :]
    wa, wb = StokesWave(H=0.04, T=1.0, d=0.5), StokesWave(H=0.02, T=1.0, d=0.5)
    vel2 = lambda xx, yy: [a - 2.0 * b for a, b in zip(wa.velocity(xx, yy, 0.2), wb.velocity(xx, yy, 0.2))]
    e = 1e-5
    uy = (vel2(x, y + e)[0] - vel2(x, y - e)[0]) / (2 * e)
    vx = (vel2(x + e, y)[1] - vel2(x - e, y)[1]) / (2 * e)
    ux = (vel2(x + e, y)[0] - vel2(x - e, y)[0]) / (2 * e)
    vy = (vel2(x, y + e)[1] - vel2(x, y - e)[1]) / (2 * e)
    scale = np.abs(vel2(x, y)[0]).max() * wa.k
    assert scale > 0
    assert np.abs(uy - vx).max() < 1e-6 * scale
    assert np.abs(ux + vy).max() < 1e-6 * scale
