"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only lays out geometry
(signed distances to flat or wavy interfaces and to boxes, marker lattices)
and draws seeded random numbers.  Everything is numpy, float64, in the
[k, j, i] (x fastest) layout of the staggered grid:

    cells (nz, ny, nx);  u (nz, ny, nx+1);  v (nz, ny+1, nx);  w (nz+1, ny, nx).

Workloads (material values of the paper's air-water examples:
rho_l = 1000, rho_g = 1.2, mu_l = 1e-3, mu_g = 1.8e-5, n_cells = 2):

* ``tank2d``  64x64 unit box, interface y = 0.5, locked 0.2x0.2 square solid
  (rho_s = 500) centred on the interface, one marker per half cell, seeded
  uniform[-1,1]*1e-2 velocity right-hand side, dt = 1e-3.
* ``tank3d``  N^3 unit box, water depth 0.6 (flat or perturbed by 8 seeded
  Fourier modes of total amplitude <= 0.05), locked 0.2x0.2x0.1 box
  (rho_s = 500) centred on the surface.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    bc: tuple = (-1.0, -1.0, -1.0, -1.0, -1.0, -1.0)
    gravity: tuple = (0.0, 0.0, -9.81)
    rho_l: float = 1000.0
    rho_g: float = 1.2
    rho_s: float = 500.0
    mu_l: float = 1e-3
    mu_g: float = 1.8e-5
    mu_s: float = 1e-3
    n_cells: float = 2.0
    theta: float = 0.5
    dt: float = 1e-3
    gravity_mode: str = "flow"
    phi: np.ndarray = None
    psi: np.ndarray = None
    markers: np.ndarray = None   # (N, 3)
    dV: float = 0.0
    lock: tuple = (True,) * 6
    box_center: tuple = None
    box_half: tuple = None
    extra: dict = field(default_factory=dict)
    open_top: bool = False       # z+ side open (zero tangential velocity, zero pressure)

    @property
    def h(self):
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)

    def cell_xyz(self):
        hx, hy, hz = self.h
        x = (np.arange(self.nx) + 0.5) * hx
        y = (np.arange(self.ny) + 0.5) * hy
        z = (np.arange(self.nz) + 0.5) * hz
        return x[None, None, :], y[None, :, None], z[:, None, None]

    def face_shape(self, c):
        s = [self.nz, self.ny, self.nx]
        s[2 - c] += 1
        return tuple(s)


def box_distance(xyz, center, half):
    """Signed distance to an axis-aligned box (negative inside)."""
    q = [np.abs(xyz[d] - center[d]) - half[d] for d in range(3)]
    q = np.broadcast_arrays(*q)
    outside = np.sqrt(sum(np.maximum(a, 0.0) ** 2 for a in q))
    inside = np.minimum(np.maximum(np.maximum(q[0], q[1]), q[2]), 0.0)
    return outside + inside


def marker_lattice(center, half, h, active=(True, True, True)):
    """Markers on a lattice of spacing h_d/2 filling a box (one per half
    cell), centred on the box.  Inactive axes get one marker layer at the
    centre.  Returns (X (N,3), dV)."""
    axes = []
    dV = 1.0
    for d in range(3):
        if active[d]:
            sp = h[d] / 2.0
            n = max(1, int(round(2.0 * half[d] / sp)))
            axes.append(center[d] + (np.arange(n) - (n - 1) / 2.0) * sp)
            dV *= sp
        else:
            axes.append(np.array([center[d]]))
            dV *= h[d]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), dV


def fourier_surface(rng, nmodes=8, amp=0.05):
    """Seeded interface perturbation eta(x, y): nmodes cosines with integer
    wave numbers 1..4 in each direction, amplitudes summing to <= amp."""
    kx = rng.integers(1, 5, size=nmodes)
    ky = rng.integers(1, 5, size=nmodes)
    a = rng.uniform(0.0, amp / nmodes, size=nmodes)
    th = rng.uniform(0.0, 2 * np.pi, size=nmodes)

    def eta(x, y):
        s = 0.0
        for m in range(nmodes):
            s = s + a[m] * np.cos(2 * np.pi * (kx[m] * x + ky[m] * y) + th[m])
        return s
    return eta


def tank2d(n=64, seed=0, with_body=True):
    c = Case(nx=n, ny=n, nz=1, lz=1.0 / n, bc=(-1.0, -1.0, -1.0, -1.0, 1.0, 1.0),
             gravity=(0.0, -9.81, 0.0), dt=1e-3)
    x, y, z = c.cell_xyz()
    c.phi = np.broadcast_to(y - 0.5, (1, n, n)).copy()
    center = (0.5, 0.5, 0.5 * c.lz)
    half = (0.1, 0.1, 0.5 * c.lz)
    if with_body:
        c.psi = np.broadcast_to(box_distance((x, y, z), center, (0.1, 0.1, 1e9)), (1, n, n)).copy()
        c.markers, c.dV = marker_lattice(center, half, c.h, active=(True, True, False))
        c.box_center, c.box_half = center, (0.1, 0.1, 1e9)
    else:
        c.psi = np.full((1, n, n), 1.0)
    rng = np.random.default_rng(seed)
    c.extra["rhs_u"] = [rng.uniform(-1.0, 1.0, size=c.face_shape(d)) * 1e-2 for d in range(3)]
    return c


def tank3d(n=128, seed=None, depth=0.6, with_body=True, dt=5e-4, nxyz=None, gravity_mode="flow"):
    nx, ny, nz = (n, n, n) if nxyz is None else nxyz
    c = Case(nx=nx, ny=ny, nz=nz, dt=dt, gravity_mode=gravity_mode)
    x, y, z = c.cell_xyz()
    if seed is None:
        c.phi = np.broadcast_to(z - depth, (nz, ny, nx)).copy()
    else:
        eta = fourier_surface(np.random.default_rng(seed))
        c.phi = np.broadcast_to(z - depth - eta(x, y), (nz, ny, nx)).copy()
    center = (0.5, 0.5, depth)
    half = (0.1, 0.1, 0.05)
    if with_body:
        c.psi = np.broadcast_to(box_distance((x, y, z), center, half), (nz, ny, nx)).copy()
        c.markers, c.dV = marker_lattice(center, half, c.h)
        c.box_center, c.box_half = center, half
    else:
        c.psi = np.full((nz, ny, nx), 1.0)
    return c


def random_faces(shape_fn, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, size=shape_fn(d)) * scale for d in range(3)]


def random_cells(shape, seed, scale=1.0):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape) * scale


def polygon_distance_xz(x, z, verts):
    """Signed distance (negative inside) to a convex polygon in the (x, z)
    plane, vertices counter-clockwise."""
    x, z = np.broadcast_arrays(x, z)
    d2 = np.full(x.shape, np.inf)
    inside = np.ones(x.shape, dtype=bool)
    n = len(verts)
    for a in range(n):
        x0, z0 = verts[a]
        x1, z1 = verts[(a + 1) % n]
        ex, ez = x1 - x0, z1 - z0
        wx, wz = x - x0, z - z0
        t = np.clip((wx * ex + wz * ez) / (ex * ex + ez * ez), 0.0, 1.0)
        dx, dz = wx - t * ex, wz - t * ez
        d2 = np.minimum(d2, dx * dx + dz * dz)
        inside &= (ex * wz - ez * wx) >= 0.0
    d = np.sqrt(d2)
    return np.where(inside, -d, d)


def wave_tank(nx=256, ny=128, nz=128, lx=4.0, ly=1.0, lz=1.0, depth=0.5, H=0.05, T=1.0, dt=0.01,
              with_bar=True):
    """Numerical wave tank: still water of depth `depth`, a second-order
    Stokes wave generated in [0, 0.5] and damped in [lx-0.5, lx], and a locked
    submerged trapezoidal bar on the bed (0.3 high, base x in [1.5, 2.5], top
    0.182 long centred at x = 2, spanning the tank), one marker per half cell.
    The bar is locked with rho_s = rho_l (Sec. 5)."""
    c = Case(nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, lz=lz, dt=dt)
    c.rho_s = c.rho_l
    x, y, z = c.cell_xyz()
    c.phi = np.broadcast_to(z - depth, (nz, ny, nx)).copy()
    verts = [(1.5, 0.0), (2.5, 0.0), (2.0 + 0.091, 0.3), (2.0 - 0.091, 0.3)]
    c.extra["wave"] = dict(H=H, T=T, depth=depth, x_gen=0.5, x_damp=lx - 0.5)
    if with_bar:
        c.psi = np.broadcast_to(polygon_distance_xz(x, z, verts), (nz, ny, nx)).copy()
        hx, hy, hz = c.h
        xs = (np.arange(int(round(1.0 / (hx / 2)))) + 0.5) * (hx / 2) + 1.5
        zs = (np.arange(int(round(0.3 / (hz / 2)))) + 0.5) * (hz / 2)
        ys = (np.arange(int(round(ly / (hy / 2)))) + 0.5) * (hy / 2)
        Xg, Zg = np.meshgrid(xs, zs, indexing="ij")
        keep = polygon_distance_xz(Xg, Zg, verts) < 0.0
        px, pz = Xg[keep], Zg[keep]
        Y = np.repeat(ys, px.size)
        c.markers = np.stack([np.tile(px, ys.size), Y, np.tile(pz, ys.size)], axis=1)
        c.dV = (hx / 2) * (hy / 2) * (hz / 2)
    else:
        c.psi = np.full((nz, ny, nx), 1.0)
    return c


def smooth_field(rng, shape, modes=6, noise=0.05):
    """Seeded smooth random cell field (z, y, x) of zero mean: a sum of
    products of cosines of low wavenumbers (0..3 per axis, Neumann-compatible)
    plus a little white noise."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                          indexing="ij")
    e = np.zeros(shape)
    for _ in range(modes):
        k = rng.integers(0, 4, size=3)
        e += rng.standard_normal() * np.cos(np.pi * k[0] * x) * np.cos(np.pi * k[1] * y) * np.cos(np.pi * k[2] * z)
    e += noise * rng.standard_normal(shape)
    return e - e.mean()


def cylinder_distance(xyz, center, radius, half_length):
    """Signed distance to a capped cylinder with its axis along y (input
    generator; the library and the oracle compute their own)."""
    x, y, z = xyz
    qr = np.sqrt((x - center[0]) ** 2 + (z - center[2]) ** 2) - radius
    qy = np.abs(y - center[1]) - half_length
    qr, qy = np.broadcast_arrays(qr, qy)
    return np.sqrt(np.maximum(qr, 0.0) ** 2 + np.maximum(qy, 0.0) ** 2) + np.minimum(np.maximum(qr, qy), 0.0)


def cylinder_lattice(center, radius, half_length, h):
    """Markers at half-cell spacing filling a cylinder along y: the points of
    the box lattice around it that lie inside.  Returns (X (N,3), dV)."""
    X, dV = marker_lattice(center, (radius, half_length, radius), h)
    r2 = (X[:, 0] - center[0]) ** 2 + (X[:, 2] - center[2]) ** 2
    return X[r2 <= radius * radius], dV


def tank_cylinder(nxyz=(32, 16, 16), lxyz=(2.0, 1.0, 1.0), seed=None, depth=0.5, radius=0.15, length=0.6,
                  dt=5e-4, rho_s=500.0):
    """Tank with a free-floating horizontal cylinder along y (config 5's body,
    scaled): axis at the still-water depth, rho_s = 500, free in surge, heave
    and pitch (x, z translation, rotation about y), the other DOFs locked."""
    nx, ny, nz = nxyz
    c = Case(nx=nx, ny=ny, nz=nz, lx=lxyz[0], ly=lxyz[1], lz=lxyz[2], dt=dt, gravity_mode="full", rho_s=rho_s)
    x, y, z = c.cell_xyz()
    if seed is None:
        c.phi = np.broadcast_to(z - depth, (nz, ny, nx)).copy()
    else:
        eta = fourier_surface(np.random.default_rng(seed))
        c.phi = np.broadcast_to(z - depth - eta(x / lxyz[0], y / lxyz[1]), (nz, ny, nx)).copy()
    center = (0.5 * lxyz[0], 0.5 * lxyz[1], depth)
    c.psi = np.broadcast_to(cylinder_distance((x, y, z), center, radius, 0.5 * length), (nz, ny, nx)).copy()
    c.markers, c.dV = cylinder_lattice(center, radius, 0.5 * length, c.h)
    c.lock = (False, True, False, True, False, True)
    c.extra["cylinder"] = (radius, 0.5 * length)
    return c
