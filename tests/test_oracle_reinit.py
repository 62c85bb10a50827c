"""Pins of the reinitialisation oracle (Sec. 4.1, the eikonal equation
marched to steady state with ENO2 differences, the subcell fix and the
Godunov Hamiltonian) against what the mathematics fixes: the signed distance
to a plane is a steady state, brute-force distances in 1-D, the kinks of a
distance function, second-order (or better) convergence to the distance
from a sphere, and the sign of the level set."""
import numpy as np
import pytest

from oracle import reinit as R
from oracle.grid import Grid


def _cells(n, l=1.0):
    return (np.arange(n) + 0.5) * (l / n)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_distance_is_steady(axis):
    """A planar signed distance normal to an axis has |grad phi| = 1 in
    every one-sided ENO2 difference, also across the Neumann walls, so the
    iteration leaves it unchanged (the subcell distances are exact for a
    linear phi)."""
    g = Grid(12, 10, 14, 1.0, 0.8, 1.3)
    x, y, z = np.meshgrid(_cells(12, 1.0), _cells(10, 0.8), _cells(14, 1.3), indexing="ij")
    coord = (x, y, z)[axis].transpose(2, 1, 0)  # [k, j, i]
    for sgn in (1.0, -1.0):
        phi0 = sgn * (coord - 0.437)
        phi = R.reinit(g, phi0, 20)
        assert np.abs(phi - phi0).max() < 1e-13


def test_1d_quadratic_is_exact():
    """phi~ = t (2 + 3 t), t = x - 0.37, has one zero in the box; the
    quadratic through its values is phi~ itself, so the subcell distances
    are exact and the steady state is the distance t to rounding."""
    n = 64
    g = Grid(n, 1, 1)
    t = _cells(n) - 0.37
    phi = R.reinit(g, (t * (2 + 3 * t))[None, None], 4 * n)
    assert np.abs(phi[0, 0] - t).max() < 1e-11


@pytest.mark.parametrize("n", [32, 64, 128])
def test_1d_brute_force_distance(n):
    """phi~ = t (1 + 4 t^2), t = x - 0.37, has the single zero x = 0.37, so
    its signed distance is x - 0.37 on every cell.  The quadratic subcell
    interpolation of a cubic is third-order accurate at the interface and
    the linear distance is carried exactly from there."""
    g = Grid(n, 1, 1)
    x = _cells(n)
    t = x - 0.37
    phi = R.reinit(g, (t * (1 + 4 * t * t))[None, None], 4 * n)
    err = np.abs(phi[0, 0] - t).max()
    assert err < 20.0 / n ** 3, err


@pytest.mark.parametrize("case", ["ridge", "valley"])
def test_kinks_of_the_distance(case):
    """Distance functions with a kink on a face: a ridge in the positive
    phase (0.25 - |x - 1/2|) and a valley in the negative one
    (|x - 1/2| - 0.3).  The Godunov upwinding takes each side's slope, so
    the steady state is exact; taking the wrong branch of the Hamiltonian at
    the kink would give |grad phi| = 1/2 there and move it."""
    n = 64
    g = Grid(n, 1, 1)
    x = _cells(n)
    if case == "ridge":
        exact = 0.25 - np.abs(x - 0.5)
        phi0 = 3.0 * exact
    else:
        exact = np.abs(x - 0.5) - 0.3
        phi0 = 2.0 * exact
    phi = R.reinit(g, phi0[None, None], 150)
    assert np.abs(phi[0, 0] - exact).max() < 1e-9


def _sphere(n):
    g = Grid(n, n, n)
    c = _cells(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    sd = np.sqrt((x - 0.51) ** 2 + (y - 0.48) ** 2 + (z - 0.5) ** 2) - 0.3
    return g, sd, sd * (1.5 + 0.5 * (x - 0.5))


def test_sphere_converges_at_second_order():
    """phi~ = (|x - c| - R) (1.5 + (x - 1/2)/2) keeps the sphere as its zero
    set but is not a distance; after 60 pseudo-time steps, in the band of
    three cells around the interface the result approaches |x - c| - R with
    the grid spacing at second order or better, and no cell changes sign."""
    errs = []
    for n in (16, 32):
        g, sd, phi0 = _sphere(n)
        phi = R.reinit(g, phi0, 60)
        band = np.abs(sd) < 3.0 / n
        errs.append(np.abs(phi - sd)[band].max())
        assert np.array_equal(np.sign(phi), np.sign(phi0))
    assert errs[0] < 1e-2, errs
    assert errs[1] < 1e-3 and errs[1] < errs[0] / 6.0, errs


def test_interface_held_where_the_gradient_nearly_vanishes():
    """The unit circle in [-2, 2]^2 given by ((x-1)^2 + (y-1)^2 + 0.1)(r - 1),
    whose gradient drops to a tenth on part of the circle: a scheme that
    lets the interface drift there stops converging to r - 1, while the
    subcell fix, which pins the interface where the quadratic through phi~
    puts it, converges at second order or better in the band of two cells."""
    errs = []
    for n in (40, 80):
        c = (np.arange(n) + 0.5) * 4.0 / n - 2.0
        y, x = np.meshgrid(c, c, indexing="ij")
        sd = np.sqrt(x * x + y * y) - 1.0
        phi = R.reinit(Grid(n, n, 1, 4.0, 4.0, 1.0), (((x - 1) ** 2 + (y - 1) ** 2 + 0.1) * sd)[None], n)
        errs.append(np.abs(phi[0] - sd)[np.abs(sd) < 8.0 / n].max())
    assert errs[1] < 2e-4 and errs[1] < errs[0] / 6.0, errs


def test_two_dimensional_equals_extruded():
    """nz = 1 is the 2-D problem: a circle there equals every z-slice of the
    z-extruded cylinder in 3-D (z derivatives of a z-independent field vanish
    through the mirror ghosts, and a z spacing no smaller than the in-plane
    one does not limit the pseudo-time step)."""
    n = 20
    c = _cells(n)
    y, x = np.meshgrid(c, c, indexing="ij")
    sd = np.sqrt((x - 0.47) ** 2 + (y - 0.52) ** 2) - 0.27
    phi0 = sd * (1.2 + x * y)
    a = R.reinit(Grid(n, n, 1, 1.0, 1.0, 0.1), phi0[None], 30)
    b = R.reinit(Grid(n, n, 5, 1.0, 1.0, 0.5), np.broadcast_to(phi0, (5, n, n)), 30)
    assert np.abs(a[0] - sd).max() < 0.02
    for k in range(5):
        assert np.abs(b[k] - a[0]).max() < 1e-14


def test_single_cell_and_zero_are_immobile():
    """A cell where phi~ is exactly zero keeps its value, and a grid of one
    cell has nothing to march."""
    g = Grid(9, 1, 1)
    x = _cells(9)
    phi0 = 2.0 * (x - 0.5)  # cell 4 sits on the interface: phi~ = 0
    phi = R.reinit(g, phi0[None, None], 300)
    assert phi[0, 0, 4] == 0.0
    assert np.abs(phi[0, 0] - (x - 0.5)).max() < 1e-12
    one = R.reinit(Grid(1, 1, 1), np.array([[[0.3]]]), 5)
    assert one[0, 0, 0] == 0.3


def test_two_cell_transient_closed_form():
    """Two cells, phi~ = a (x - 1/2): each cell's only active difference is
    the subcell one across the interface at h/2, so a forward-Euler stage
    maps the error e = phi_0 + 1/4 to (1 - cfl) e (local step cfl h/2 over
    the distance h/2), and the two-stage TVD Runge-Kutta step to
    (1 + (1 - cfl)^2)/2 e: 0.745 e for cfl = 0.3."""
    a, m = 3.0, 5
    phi = R.reinit(Grid(2, 1, 1), np.array([[[-a / 4, a / 4]]]), m)
    e = (0.25 - a / 4) * (0.5 * (1 + 0.7 ** 2)) ** m
    assert phi[0, 0, 0] == pytest.approx(-0.25 + e, rel=1e-14)
    assert phi[0, 0, 1] == pytest.approx(0.25 - e, rel=1e-14)
