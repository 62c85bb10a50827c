"""Material properties from the two level sets (Sec. 4.1 and Sec. 5).

Oracle (test infrastructure only).

* smoothed Heaviside over n_cells cells on either side of an interface
  (Sec. 4.1, smoothed-Heaviside equation);
* two-stage property: flow phase from phi, then the solid from psi
  (Sec. 4.1, the flow-phase and whole-domain property equations);
* viscosity at cell centres, harmonic average onto edges (Sec. 4.2,
  footnote to step 1 of the time-stepping scheme);
* face density from level sets averaged onto faces (Sec. 4.2.2, the
  "level set synchronized density field");
* flow-only density rho^flow for the well-balanced gravity force (Sec. 5).

Reading: the paper assumes hx = hy = hz for the transition width
n_cells*dx; for unequal spacing the width uses the geometric mean of the
active spacings, by analogy with the sqrt(dV) rule of Sec. 7.1.
"""
import numpy as np

from .grid import Grid


def char_spacing(g: Grid):
    """Characteristic grid spacing for the Heaviside width."""
    if g.dim == 2:
        return float(np.sqrt(g.hx * g.hy))
    return float((g.hx * g.hy * g.hz) ** (1.0 / 3.0))


def heaviside(phi, eps):
    """Smoothed Heaviside of Sec. 4.1: 0 below -eps, 1 above +eps, and
    (1 + phi/eps + sin(pi phi/eps)/pi)/2 in between."""
    phi = np.asarray(phi, dtype=np.float64)
    mid = 0.5 * (1.0 + phi / eps + np.sin(np.pi * phi / eps) / np.pi)
    return np.where(phi < -eps, 0.0, np.where(phi > eps, 1.0, mid))


def two_stage(phi, psi, z_l, z_g, z_s, eps):
    """Flow phase from phi (liquid where phi<0), then solid where psi<0."""
    z_flow = z_l + (z_g - z_l) * heaviside(phi, eps)
    return z_s + (z_flow - z_s) * heaviside(psi, eps)


def flow_only(phi, z_l, z_g, eps):
    return z_l + (z_g - z_l) * heaviside(phi, eps)


def face_average(g: Grid, a, c):
    """Arithmetic mean of the two cells sharing each c-face; a wall face takes
    its single interior neighbour (Neumann mirror ghost)."""
    ap = np.take(a, [0], axis=a.ndim - 1 - c)
    aq = np.take(a, [-1], axis=a.ndim - 1 - c)
    ext = np.concatenate([ap, a, aq], axis=a.ndim - 1 - c)
    ax = ext.ndim - 1 - c
    n = ext.shape[ax]
    lo = np.take(ext, np.arange(0, n - 1), axis=ax)
    hi = np.take(ext, np.arange(1, n), axis=ax)
    return 0.5 * (lo + hi)


def edge_harmonic(g: Grid, mu_cc, c1, c2):
    """Harmonic mean of the four cells around each edge lying in the (c1,c2)
    plane, i.e. the edge at (i h_c1, j h_c2) running along the third axis.
    Ghost cells beyond walls are Neumann mirrors, so an edge on a wall takes
    the harmonic mean of its two interior cells (each counted twice)."""
    from .grid import pad_cell_neumann
    m = pad_cell_neumann(mu_cc)
    inv = 1.0 / m
    a1 = m.ndim - 1 - c1
    a2 = m.ndim - 1 - c2
    # keep the third axis unpadded
    c3 = 3 - c1 - c2
    a3 = m.ndim - 1 - c3
    n3 = inv.shape[a3]
    inv = np.take(inv, np.arange(1, n3 - 1), axis=a3)
    n1 = inv.shape[a1]
    n2 = inv.shape[a2]
    s = 0.0
    for o1 in (0, 1):
        for o2 in (0, 1):
            t = np.take(inv, np.arange(o1, n1 - 1 + o1), axis=a1)
            t = np.take(t, np.arange(o2, n2 - 1 + o2), axis=a2)
            s = s + t
    return 4.0 / s


class Materials:
    """Every coefficient the Stokes operator and the step need."""

    def __init__(self, g: Grid, phi, psi, rho_l, rho_g, rho_s, mu_l, mu_g, mu_s, n_cells=2.0):
        eps = n_cells * char_spacing(g)
        self.eps = eps
        self.rho_cc = two_stage(phi, psi, rho_l, rho_g, rho_s, eps)
        self.mu_cc = two_stage(phi, psi, mu_l, mu_g, mu_s, eps)
        self.rho_face = []
        self.rho_flow_face = []
        for c in range(3):
            phf = face_average(g, phi, c)
            psf = face_average(g, psi, c)
            self.rho_face.append(two_stage(phf, psf, rho_l, rho_g, rho_s, eps))
            self.rho_flow_face.append(flow_only(phf, rho_l, rho_g, eps))
        self.mu_xy = edge_harmonic(g, self.mu_cc, 0, 1)
        self.mu_xz = edge_harmonic(g, self.mu_cc, 0, 2)
        self.mu_yz = edge_harmonic(g, self.mu_cc, 1, 2)
