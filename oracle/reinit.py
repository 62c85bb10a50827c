"""Reinitialisation of the flow level set (Sec. 4.1, the eikonal equation).

Oracle (test infrastructure only).

After advection the flow level set phi~ is brought back to a signed
distance by marching the Hamilton-Jacobi equation

    d phi / d tau + sgn(phi~) (|grad phi| - 1) = 0,   phi(tau = 0) = phi~

towards its steady state |grad phi| = 1.  The paper names the ingredients
of its discretisation and leaves the details to its references; this module
follows those published methods, in this order, on the cell-centred grid:

1. one-sided second-order ENO differences along each axis,
       D+ phi_i = (phi_{i+1} - phi_i)/h - (h/2) minmod(Dxx phi_i, Dxx phi_{i+1}),
       D- phi_i = (phi_i - phi_{i-1})/h + (h/2) minmod(Dxx phi_i, Dxx phi_{i-1}),
   Dxx phi_i = (phi_{i+1} - 2 phi_i + phi_{i-1})/h^2, minmod(a, b) = 0 when
   a and b differ in sign, else the one of smaller magnitude;
2. the subcell fix (Min 2010): where phi~ changes sign between cell i and
   its neighbour, the interface lies at distance h+ (h-) from x_i, taken as
   the root inside the cell interval of the quadratic through phi~_i and
   phi~_{i+1} with second difference minmod(Dxx phi~_i, Dxx phi~_{i+1}), and
   the difference across it uses the interface value 0:
       D+ phi_i = (0 - phi_i)/h+ - (h+/2) minmod(Dxx phi_i, Dxx phi_{i+1})
   (and the mirror form for D-);
3. the Godunov Hamiltonian of sgn(phi~):
       s > 0:  |grad phi|^2 = sum_d max(max(D-, 0)^2, min(D+, 0)^2)
       s < 0:  |grad phi|^2 = sum_d max(min(D-, 0)^2, max(D+, 0)^2);
4. two-stage TVD Runge-Kutta in pseudo-time with the local step
   dtau_i = cfl * min(h_d over the axes with more than one cell, every h+-
   of cell i), the classical choice of the subcell-fix literature so that
   cells next to the interface stay stable.

The interface is immobile (Son 2005): sgn(phi~) and the subcell distances
come from phi~ and stay fixed during the iteration, and a cell where phi~ is
exactly zero keeps its value.  Cell-centred values take homogeneous Neumann
(mirror) ghosts, as in the advection.  Each call runs a fixed number of
pseudo-time iterations; the paper reinitialises every time step and does not
state its stopping rule.

Parity: pinned (exact invariance of planar signed distances, brute-force
1-D distances, exactness for a quadratic profile, kinks of the distance
function, second-order convergence to the distance from a sphere and to a
circle whose level-set gradient nearly vanishes, sign preservation).  The
mirror-ghost convention leaves all of these steady states unchanged; the GPU
parity tests hold the kernels to it.
"""
import numpy as np

from .grid import Grid

CFL = 0.3


def _minmod(a, b):
    return np.where(a * b > 0.0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _mirror_take(q, d, offset):
    """q shifted by `offset` cells along axis d with Neumann mirror ghosts:
    element i of the result is q at cell i + offset (ghost -1 <-> cell 0,
    ghost -2 <-> cell 1, and the same at the upper side)."""
    ax = q.ndim - 1 - d
    n = q.shape[ax]
    ids = []
    for i in range(n):
        m = i + offset
        if m < 0:
            m = -m - 1
        elif m >= n:
            m = 2 * n - 1 - m
        ids.append(min(max(m, 0), n - 1))
    return np.take(q, ids, axis=ax)


def _interface_distance(a, b, c):
    """Distance, in units of the cell spacing, from the centre holding `a` to
    the zero of the quadratic through a (at 0) and b (at 1) whose second
    difference is c, for a * b < 0.  In the local coordinate t = xi - 1/2 the
    quadratic is c0 + c1 t + c2 t^2 with c2 = c/2, c1 = b - a,
    c0 = (a + b)/2 - c/8; the zero inside [-1/2, 1/2] is the root of smaller
    magnitude, t = -2 c0 / (c1 + sgn(c1) sqrt(c1^2 - 4 c2 c0)), which reduces
    to the linear zero when c = 0."""
    c2 = 0.5 * c
    c1 = b - a
    c0 = 0.5 * (a + b) - 0.125 * c
    disc = np.maximum(c1 * c1 - 4.0 * c2 * c0, 0.0)
    t = -2.0 * c0 / (c1 + np.sign(c1) * np.sqrt(disc))
    return 0.5 + t


def one_sided(g: Grid, phi, phi0, d):
    """ENO2 one-sided differences D-, D+ of phi along axis d with the subcell
    fix from phi0 (steps 1 and 2), and the smallest interface distance of each
    cell along d (h_d where phi0 does not change sign)."""
    h = g.h[d]
    p = {o: _mirror_take(phi, d, o) for o in (-2, -1, 0, 1, 2)}
    q = {o: _mirror_take(phi0, d, o) for o in (-2, -1, 0, 1, 2)}
    pxx = {o: p[o - 1] - 2.0 * p[o] + p[o + 1] for o in (-1, 0, 1)}  # undivided
    qxx = {o: q[o - 1] - 2.0 * q[o] + q[o + 1] for o in (-1, 0, 1)}
    mp = _minmod(pxx[0], pxx[1])
    mm = _minmod(pxx[0], pxx[-1])
    Dp = (p[1] - p[0]) / h - 0.5 * mp / h
    Dm = (p[0] - p[-1]) / h + 0.5 * mm / h
    hloc = np.full(phi.shape, h)
    with np.errstate(divide="ignore", invalid="ignore"):
        cross_p = q[0] * q[1] < 0.0
        hp = h * _interface_distance(q[0], q[1], _minmod(qxx[0], qxx[1]))
        hp = np.where(cross_p, np.clip(hp, 1e-10 * h, h), h)
        Dp = np.where(cross_p, (0.0 - p[0]) / hp - 0.5 * hp * mp / (h * h), Dp)
        cross_m = q[0] * q[-1] < 0.0
        hm = h * _interface_distance(q[0], q[-1], _minmod(qxx[0], qxx[-1]))
        hm = np.where(cross_m, np.clip(hm, 1e-10 * h, h), h)
        Dm = np.where(cross_m, (p[0] - 0.0) / hm + 0.5 * hm * mm / (h * h), Dm)
    hloc = np.minimum(hloc, np.minimum(hp, hm))
    return Dm, Dp, hloc


def rate(g: Grid, phi, phi0, cfl=CFL):
    """-sgn(phi0) (|grad phi|_Godunov - 1) and the local pseudo-time step
    (steps 3 and 4)."""
    s = np.sign(phi0)
    grad2 = np.zeros(phi.shape)
    dtau = np.full(phi.shape, np.inf)
    ns = (g.nx, g.ny, g.nz)
    for d in range(3):
        if ns[d] == 1:
            continue  # no neighbours along this axis: the derivative vanishes
        Dm, Dp, hloc = one_sided(g, phi, phi0, d)
        pos = np.maximum(np.maximum(Dm, 0.0) ** 2, np.minimum(Dp, 0.0) ** 2)
        neg = np.maximum(np.minimum(Dm, 0.0) ** 2, np.maximum(Dp, 0.0) ** 2)
        grad2 += np.where(s > 0, pos, neg)
        dtau = np.minimum(dtau, cfl * hloc)
    dtau = np.where(np.isfinite(dtau), dtau, 0.0)  # a single cell: nothing to march
    return -s * (np.sqrt(grad2) - 1.0), dtau


def reinit(g: Grid, phi0, iters, cfl=CFL):
    """`iters` two-stage TVD Runge-Kutta pseudo-time steps from phi0."""
    phi0 = np.asarray(phi0, dtype=np.float64)
    phi = phi0.copy()
    for _ in range(iters):
        L, dtau = rate(g, phi, phi0, cfl)
        p1 = phi + dtau * L
        L1, _ = rate(g, p1, phi0, cfl)
        phi = 0.5 * phi + 0.5 * (p1 + dtau * L1)
    return phi
