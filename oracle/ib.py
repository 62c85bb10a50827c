"""Lagrangian-Eulerian transfer with the IB4 kernel (Sec. 3.3).

Oracle (test infrastructure only).

Interpolation  U_l = sum_faces u_f delta_h(x_f - X_l) hx hy hz
Spreading      f_f = sum_l F_l delta_h(x_f - X_l) dV_l
with delta_h(x) = prod_d phi4(x_d / h_d) / h_d and phi4 Peskin's four-point
kernel (Sec. 3.3.1 cites it without printing it; the formula below is the
published one, restated from its defining moment conditions' solution):

    phi4(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8     |r| <= 1
            = (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8    1 <= |r| <= 2
            = 0                                            otherwise

Near walls (Sec. 3.3.2): J_BC fills ghost values from the boundary condition
and then uses the standard weights; S_BC spreads into ghosts and adds each
ghost's value back onto its mirror image, so that S_BC is the adjoint of
J_BC.  Ghost rules: a tangential component mirrors with the wall's sign s
(-1 no-slip, +1 free-slip); the normal component is odd about the wall face
(whose own value is zero, so taps landing on it drop out).
"""
import numpy as np

from .grid import Grid


def phi4(r):
    r = np.abs(np.asarray(r, dtype=np.float64))
    inner = (3.0 - 2.0 * r + np.sqrt(np.maximum(1.0 + 4.0 * r - 4.0 * r * r, 0.0))) / 8.0
    outer = (5.0 - 2.0 * r - np.sqrt(np.maximum(-7.0 + 12.0 * r - 4.0 * r * r, 0.0))) / 8.0
    return np.where(r <= 1.0, inner, np.where(r <= 2.0, outer, 0.0))


def _map_index(i, n, normal, s_lo, s_hi):
    """Map tap indices along one axis to stored indices and signs.

    normal: the axis is the component's own direction (stored faces 0..n,
    faces 0 and n are walls with value 0).  Otherwise stored cells 0..n-1.
    Returns (index, sign, valid)."""
    i = np.array(i, dtype=np.int64)
    sgn = np.ones(i.shape)
    for _ in range(8):  # repeated reflections only matter for n = 1
        if normal:
            lo = i < 0
            i = np.where(lo, -i, i)
            sgn = np.where(lo, -sgn, sgn)
            hi = i > n
            i = np.where(hi, 2 * n - i, i)
            sgn = np.where(hi, -sgn, sgn)
        else:
            lo = i < 0
            i = np.where(lo, -1 - i, i)
            sgn = np.where(lo, s_lo * sgn, sgn)
            hi = i >= n
            i = np.where(hi, 2 * n - 1 - i, i)
            sgn = np.where(hi, s_hi * sgn, sgn)
    if normal:
        valid = (i > 0) & (i < n)
    else:
        valid = (i >= 0) & (i < n)
    return i, sgn, valid


def _taps(g: Grid, X, c):
    """For component c and markers X (N,3): per axis, 4 stored indices,
    signs, validity and kernel weights (each array (N,4))."""
    n = (g.nx, g.ny, g.nz)
    out = []
    for d in range(3):
        h = g.h[d]
        normal = d == c
        xs = X[:, d] / h if normal else X[:, d] / h - 0.5
        base = np.floor(xs).astype(np.int64) - 1
        idx = base[:, None] + np.arange(4)[None, :]
        r = idx - xs[:, None]
        w = phi4(r)
        mi, sg, ok = _map_index(idx, n[d], normal, g.sign(d, 0), g.sign(d, 1))
        out.append((mi, sg, ok, w))
    return out


def interpolate(g: Grid, vel, X):
    """J_BC u: velocity (u, v, w) -> marker velocities (N,3)."""
    N = X.shape[0]
    U = np.zeros((N, 3))
    for c in range(3):
        q = vel[c]
        (ix, sx, okx, wx), (iy, sy, oky, wy), (iz, sz, okz, wz) = _taps(g, X, c)
        for a in range(4):
            for b in range(4):
                for e in range(4):
                    ok = okx[:, a] & oky[:, b] & okz[:, e]
                    wt = wx[:, a] * wy[:, b] * wz[:, e] * sx[:, a] * sy[:, b] * sz[:, e]
                    k = np.where(ok, iz[:, e], 0)
                    j = np.where(ok, iy[:, b], 0)
                    i = np.where(ok, ix[:, a], 0)
                    U[:, c] += np.where(ok, wt * q[k, j, i], 0.0)
    return U


def spread(g: Grid, F, X, dV):
    """S_BC F: marker values F (N,3) with volumes dV -> face arrays."""
    hx, hy, hz = g.h
    out = [np.zeros(g.face_shape(c)) for c in range(3)]
    scale = dV / (hx * hy * hz)
    for c in range(3):
        (ix, sx, okx, wx), (iy, sy, oky, wy), (iz, sz, okz, wz) = _taps(g, X, c)
        for a in range(4):
            for b in range(4):
                for e in range(4):
                    ok = okx[:, a] & oky[:, b] & okz[:, e]
                    wt = wx[:, a] * wy[:, b] * wz[:, e] * sx[:, a] * sy[:, b] * sz[:, e]
                    val = wt * F[:, c] * scale
                    np.add.at(out[c], (iz[ok, e], iy[ok, b], ix[ok, a]), val[ok])
    return out
