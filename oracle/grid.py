"""Staggered MAC grid of Sec. 3.1 (Eulerian discretization).

Oracle (test infrastructure only).

Cells (i, j, k), i = 0..nx-1, centred at ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz).
Arrays are numpy arrays indexed [k, j, i] (x fastest in memory), with any
number of leading batch axes allowed by every operator:

    cell scalar  (nz,   ny,   nx)     p, phi, psi, rho_cc, mu_cc
    u  x-faces   (nz,   ny,   nx+1)   u[k,j,i] at (i hx, (j+1/2)hy, (k+1/2)hz)
    v  y-faces   (nz,   ny+1, nx)     v[k,j,i] at ((i+1/2)hx, j hy, (k+1/2)hz)
    w  z-faces   (nz+1, ny,   nx)     w[k,j,i] at ((i+1/2)hx, (j+1/2)hy, k hz)
    mu_xy edges  (nz,   ny+1, nx+1)   at (i hx, j hy, (k+1/2)hz)
    mu_xz edges  (nz+1, ny,   nx+1)   at (i hx, (j+1/2)hy, k hz)
    mu_yz edges  (nz+1, ny+1, nx)     at ((i+1/2)hx, j hy, k hz)

Walls.  Every side of the box is a wall.  Faces lying on a wall carry the
normal velocity, which is zero there; they are stored but are not unknowns
(every operator writes 0 on them).  Tangential velocity ghosts across a wall
are  u_ghost = s * u_interior  with s = -1 for no-slip and s = +1 for
free-slip.  Cell-centred scalars (phi, psi, rho, mu, p) take homogeneous
Neumann ghosts (mirror copies).

Open top (Sec. 7.1's wave tank: zero tangential velocity and zero pressure on
the top boundary).  With open_top the z+ side is not a wall: its tangential
velocity ghosts take s = -1 (bc[5] must be NO_SLIP), the w-faces on it are
unknowns, the pressure ghost above it is -p of the cell below (p = 0 on the
plane, linear across it), and the ghost of w above it is the mirror image
w[nz+1] = w[nz-1] (a zero normal derivative: the tangential velocity and
hence its tangential derivatives vanish on the plane, so continuity leaves
dw/dz = 0 there).

Two-dimensional problems (Sec. 3 says the 2-D discretization is analogous)
are run as nz = 1 with free-slip walls in z: every z-derivative then vanishes
identically and all w-faces are wall faces.
"""
from dataclasses import dataclass, field

import numpy as np

NO_SLIP = -1.0
FREE_SLIP = 1.0


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    # tangential-ghost sign per side: (x-, x+, y-, y+, z-, z+)
    bc: tuple = field(default=(NO_SLIP,) * 6)
    # z+ side open (zero tangential velocity, zero pressure)
    open_top: bool = False

    def __post_init__(self):
        if self.open_top and (self.bc[5] != NO_SLIP or self.nz < 2):
            raise ValueError("an open top needs bc[5] = NO_SLIP and nz >= 2")

    @property
    def h(self):
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)

    @property
    def hx(self):
        return self.lx / self.nx

    @property
    def hy(self):
        return self.ly / self.ny

    @property
    def hz(self):
        return self.lz / self.nz

    @property
    def dim(self):
        return 2 if self.nz == 1 else 3

    @property
    def cell_shape(self):
        return (self.nz, self.ny, self.nx)

    def face_shape(self, c):
        s = [self.nz, self.ny, self.nx]
        s[2 - c] += 1
        return tuple(s)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    def n_faces(self, c):
        return int(np.prod(self.face_shape(c)))

    # --- coordinates -----------------------------------------------------
    def cell_centers(self):
        """(x, y, z) broadcastable coordinate arrays of cell centres."""
        hx, hy, hz = self.h
        x = (np.arange(self.nx) + 0.5) * hx
        y = (np.arange(self.ny) + 0.5) * hy
        z = (np.arange(self.nz) + 0.5) * hz
        return x[None, None, :], y[None, :, None], z[:, None, None]

    def face_centers(self, c):
        """Coordinates of the c-faces (c = 0 x, 1 y, 2 z)."""
        hx, hy, hz = self.h
        n = (self.nx, self.ny, self.nz)
        hs = (hx, hy, hz)
        coords = []
        for d in range(3):
            if d == c:
                a = np.arange(n[d] + 1) * hs[d]
            else:
                a = (np.arange(n[d]) + 0.5) * hs[d]
            coords.append(a)
        x, y, z = coords
        return x[None, None, :], y[None, :, None], z[:, None, None]

    def interior_face_mask(self, c):
        """True on faces that are unknowns (not lying on a wall)."""
        m = np.ones(self.face_shape(c), dtype=bool)
        ax = 2 - c
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = 0
        sl1[ax] = -1
        m[tuple(sl0)] = False
        if not (c == 2 and self.open_top):
            m[tuple(sl1)] = False
        return m

    def sign(self, axis, side):
        """Tangential ghost sign on wall (axis 0 x / 1 y / 2 z, side 0 lo / 1 hi)."""
        return self.bc[2 * axis + side]

    # --- Stokes vectors: (u, v, w, p) flattened and concatenated ----------
    def sizes(self):
        return (self.n_faces(0), self.n_faces(1), self.n_faces(2), self.n_cells)

    def pack(self, u, v, w, p):
        return np.concatenate([u.reshape(u.shape[:-3] + (-1,)),
                               v.reshape(v.shape[:-3] + (-1,)),
                               w.reshape(w.shape[:-3] + (-1,)),
                               p.reshape(p.shape[:-3] + (-1,))], axis=-1)

    def unpack(self, x):
        s = self.sizes()
        o = np.cumsum((0,) + s)
        lead = x.shape[:-1]
        u = x[..., o[0]:o[1]].reshape(lead + self.face_shape(0))
        v = x[..., o[1]:o[2]].reshape(lead + self.face_shape(1))
        w = x[..., o[2]:o[3]].reshape(lead + self.face_shape(2))
        p = x[..., o[3]:o[4]].reshape(lead + self.cell_shape)
        return u, v, w, p

    def unknown_mask(self):
        """Mask over a packed Stokes vector: True where the entry is an unknown."""
        return np.concatenate([self.interior_face_mask(0).ravel(),
                               self.interior_face_mask(1).ravel(),
                               self.interior_face_mask(2).ravel(),
                               np.ones(self.n_cells, dtype=bool)])


def pad_cell_neumann(a):
    """One mirror-ghost layer on every side of a cell array (homogeneous Neumann)."""
    pad = [(0, 0)] * (a.ndim - 3) + [(1, 1)] * 3
    return np.pad(a, pad, mode="edge")


def pad_tangential(g, q, c):
    """Ghost layer for velocity component c (0 u, 1 v, 2 w) across the walls
    tangential to it: one layer on both sides of each axis other than c, filled
    with s * (adjacent interior value).  Returns the padded array (axis c is
    not padded)."""
    out = q
    for d in range(3):
        if d == c:
            continue
        ax = out.ndim - 1 - d
        lo = np.take(out, [0], axis=ax) * g.sign(d, 0)
        hi = np.take(out, [-1], axis=ax) * g.sign(d, 1)
        out = np.concatenate([lo, out, hi], axis=ax)
    return out
