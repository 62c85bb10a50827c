"""Second-order Stokes waves and relaxation zones of the numerical wave tank
(Sec. 7.1).

Oracle (test infrastructure only).

Wave of height H and period T over still-water depth d, vertical coordinate
y measured from the still-water level (the paper's frame has the bottom at
y = -d; in the 3-D tank with its bottom at z = 0, y = z - d):

  omega^2 = g k tanh(k d)                          (dispersion relation)
  eta  = H/2 cos(th) + pi H^2/(8 lam) cosh(kd)(2 + cosh 2kd)/sinh^3(kd) cos(2 th)
  u_w  = H g k/(2 omega) cosh(k(d+y))/cosh(kd) cos(th)
         + 3 H^2 omega k/16 cosh(2k(d+y))/sinh^4(kd) cos(2 th)
  v_w  = H g k/(2 omega) sinh(k(d+y))/cosh(kd) sin(th)
         + 3 H^2 omega k/16 sinh(2k(d+y))/sinh^4(kd) sin(2 th)
  th = k x - omega t,  lam = 2 pi / k.

Relaxation at the end of each step: q <- alpha q + (1 - alpha) q_target with
alpha = 1 - (exp(xb^3.5) - 1)/(e - 1), xb the normalised distance into the
zone (0 where the zone meets the computed region, 1 at the far wall).

Dirichlet inlet (Sec. 7.1, the inlet's boundary-Heaviside equation): on the
x- plane the normal velocity of face (j, k) is (1 - H~(phi_b)) u_w(0, y_k, t)
with phi_b = y_k - eta(0, t) at the face centre, and the tangential
(vertical) velocity of the x- edge at height y_k = k h - d is
(1 - H~(phi_b)) v_w(0, y_k, t) with phi_b at the edge; H~ has the width
n_cells times the characteristic spacing of the Heaviside of the materials
(sqrt(dx dy) in 2-D, the paper's sqrt(dV); the cube root of the cell volume
in 3-D).  The span-wise velocity there is zero.  The data are taken at the
time of the velocity they bound (t^{n+1} for the implicit solve).

Readings (the paper uses a Dirichlet inlet and a damping zone only):
* the generation zone mirrors the damping zone at the inlet end; its
  targets are the level set phi = y - eta(x, t) and the liquid-only
  velocity (1 - H~(phi_target)) (u_w, v_w) (the inlet condition's form);
* damping-zone targets are still water: phi = y, u = 0;
* the transverse (span-wise) velocity is relaxed to 0 in both zones;
* the targets are evaluated at t^{n+1}.
"""
import numpy as np

from .grid import Grid
from .materials import heaviside, char_spacing


def wavenumber(omega, d, g=9.81, tol=1e-15, maxit=100):
    """Solve omega^2 = g k tanh(k d) for k by Newton's method from the
    deep-water guess k0 = omega^2 / g."""
    k = omega * omega / g
    for _ in range(maxit):
        f = g * k * np.tanh(k * d) - omega * omega
        df = g * np.tanh(k * d) + g * k * d / np.cosh(k * d) ** 2
        dk = f / df
        k -= dk
        if abs(dk) < tol * k:
            break
    return k


class StokesWave:
    def __init__(self, H, T, d, g=9.81):
        self.H, self.T, self.d, self.g = H, T, d, g
        self.omega = 2.0 * np.pi / T
        self.k = wavenumber(self.omega, d, g)
        self.lam = 2.0 * np.pi / self.k

    def eta(self, x, t):
        H, k, d, w = self.H, self.k, self.d, self.omega
        th = k * x - w * t
        c2 = np.pi * H * H / (8.0 * self.lam) * np.cosh(k * d) * (2.0 + np.cosh(2 * k * d)) / np.sinh(k * d) ** 3
        return 0.5 * H * np.cos(th) + c2 * np.cos(2 * th)

    def velocity(self, x, y, t):
        """(u_w, v_w) at horizontal position x and height y above still water."""
        H, k, d, w, g = self.H, self.k, self.d, self.omega, self.g
        th = k * x - w * t
        a1 = H * g * k / (2.0 * w) / np.cosh(k * d)
        a2 = 3.0 * H * H * w * k / 16.0 / np.sinh(k * d) ** 4
        u = a1 * np.cosh(k * (d + y)) * np.cos(th) + a2 * np.cosh(2 * k * (d + y)) * np.cos(2 * th)
        v = a1 * np.sinh(k * (d + y)) * np.sin(th) + a2 * np.sinh(2 * k * (d + y)) * np.sin(2 * th)
        return u, v


def alpha(xb):
    xb = np.clip(xb, 0.0, 1.0)
    return 1.0 - (np.exp(xb ** 3.5) - 1.0) / (np.e - 1.0)


class Zones:
    """Generation zone [0, x_gen] and damping zone [x_damp, lx] along x;
    vertical axis `vert` (2 for the 3-D tank), still-water depth d."""

    def __init__(self, wave: StokesWave, x_gen, x_damp, lx, vert=2):
        self.wave, self.x_gen, self.x_damp, self.lx, self.vert = wave, x_gen, x_damp, lx, vert

    def weights(self, x):
        """(alpha, in_gen, in_damp) at positions x (x_gen = 0: no
        generation zone, as with a Dirichlet inlet)."""
        a = np.ones_like(x, dtype=np.float64)
        gen = x < self.x_gen
        dmp = x > self.x_damp
        if self.x_gen > 0:
            a = np.where(gen, alpha((self.x_gen - x) / self.x_gen), a)
        a = np.where(dmp, alpha((x - self.x_damp) / (self.lx - self.x_damp)), a)
        return a, gen, dmp

    def relax(self, g: Grid, vel, phi, t, n_cells=2.0):
        """Relaxed copies of (u, v, w) and phi at time t."""
        d = self.wave.d
        eps = n_cells * char_spacing(g)
        out = []
        for c in range(3):
            X = np.broadcast_arrays(*g.face_centers(c))
            x = X[0]
            y = X[self.vert] - d
            a, gen, _ = self.weights(x)
            if c == 0 or c == self.vert:
                phit = y - self.wave.eta(x, t)
                uw, vw = self.wave.velocity(x, y, t)
                liquid = 1.0 - heaviside(phit, eps)
                tgt_gen = liquid * (uw if c == 0 else vw)
            else:
                tgt_gen = np.zeros_like(x)
            tgt = np.where(gen, tgt_gen, 0.0)
            q = a * vel[c] + (1.0 - a) * tgt
            q = np.where(g.interior_face_mask(c), q, vel[c])  # boundary faces keep their values
            out.append(q)
        Xc = np.broadcast_arrays(*g.cell_centers())
        x = Xc[0]
        y = Xc[self.vert] - d
        a, gen, _ = self.weights(x)
        tgt = np.where(gen, y - self.wave.eta(x, t), y)
        return out, a * phi + (1.0 - a) * tgt


class Inlet:
    """Dirichlet wave inlet on the x- plane (Sec. 7.1) of a tank whose
    vertical axis is z; still-water depth d = wave.d."""

    def __init__(self, wave: StokesWave):
        self.wave = wave

    def _liquid(self, g: Grid, y, t, n_cells):
        phib = y - self.wave.eta(0.0, t)
        return 1.0 - heaviside(phib, n_cells * char_spacing(g))

    def normal(self, g: Grid, t, n_cells=2.0):
        """u on the x- faces, shape (nz, ny)."""
        _, _, z = g.face_centers(0)
        yy = z[..., 0] - self.wave.d
        uw, _ = self.wave.velocity(0.0, yy, t)
        out = self._liquid(g, yy, t, n_cells) * uw
        return np.broadcast_to(out, (g.nz, g.ny)).copy()

    def tangential(self, g: Grid, t, n_cells=2.0):
        """w on the x- edges (heights k hz), shape (nz+1, ny)."""
        yy = np.arange(g.nz + 1)[:, None] * g.hz - self.wave.d
        _, vw = self.wave.velocity(0.0, yy, t)
        out = self._liquid(g, yy, t, n_cells) * vw
        return np.broadcast_to(out, (g.nz + 1, g.ny)).copy()
