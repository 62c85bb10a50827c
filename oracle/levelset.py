"""Level-set advection (Sec. 4.2.1) and the structure level set (Sec. 4.1).

Oracle (test infrastructure only).

  phi^{n+1,k+1} = phi^n - dt Q(u^{n+1/2,k}, phi^{n+1/2,k})

with Q the conservative flux divergence div(u phi) on cell centres, face
values of phi limited by the same bounded cubic-upwind (CUI) scheme used for
the momentum transport.  Reading: the paper's Q is an xsPPM7-limited
piecewise-parabolic scheme that it does not print; the CUI limiter stands in
for it.  Homogeneous Neumann ghosts for phi on every wall; faces on walls
carry zero velocity and hence zero flux.  No reinitialisation is applied.

The structure level set is rebuilt every cycle from the markers' centre of
mass as an analytic signed distance (Sec. 4.1): for a box of half-extents
a about centre X_c,  q = |x - X_c| - a,  psi = |max(q, 0)| + min(max_d q_d, 0).
"""
import numpy as np

from .grid import Grid
from .transport import cui


def _extend_even(q, d):
    ax = q.ndim - 1 - d
    n = q.shape[ax]
    ids = [min(max(i, 0), n - 1) for i in (1, 0)] + list(range(n)) + \
          [min(max(i, 0), n - 1) for i in (n - 1, n - 2)]
    return np.take(q, ids, axis=ax)


def advect(g: Grid, vel, phi_n, phi_half, dt):
    Q = np.zeros(g.cell_shape)
    for d in range(3):
        e = _extend_even(phi_half, d)
        ax = e.ndim - 1 - d
        n = phi_half.shape[phi_half.ndim - 1 - d]
        cnt = n + 1  # faces 0..n; face m between cells m-1 and m

        def take(off):
            return np.take(e, np.arange(off, off + cnt), axis=ax)

        qm2, qm1, q0, q1 = take(0), take(1), take(2), take(3)
        a = vel[d]
        lim = np.where(a > 0.0, cui(qm2, qm1, q0), cui(q1, q0, qm1))
        F = a * lim
        axf = F.ndim - 1 - d
        nf = F.shape[axf]
        Q += (np.take(F, np.arange(1, nf), axis=axf) - np.take(F, np.arange(0, nf - 1), axis=axf)) / g.h[d]
    return phi_n - dt * Q


def cylinder_sdf(g: Grid, center, radius, half_length):
    """Signed distance to a solid circular cylinder with its axis along y,
    capped at |y - y_c| = half_length (Sec. 4.1: psi is the analytic signed
    distance of the body about its centre of mass).  Outside: the Euclidean
    distance to the closed cylinder; inside: minus the distance to the
    nearest of the mantle and the two caps."""
    x, y, z = g.cell_centers()
    qr = np.sqrt((x - center[0]) ** 2 + (z - center[2]) ** 2) - radius
    qy = np.abs(y - center[1]) - half_length
    qr, qy = np.broadcast_arrays(qr, qy)
    outside = np.sqrt(np.maximum(qr, 0.0) ** 2 + np.maximum(qy, 0.0) ** 2)
    inside = np.minimum(np.maximum(qr, qy), 0.0)
    return outside + inside


def box_sdf(g: Grid, center, half):
    x, y, z = g.cell_centers()
    q = [np.abs(x - center[0]) - half[0], np.abs(y - center[1]) - half[1], np.abs(z - center[2]) - half[2]]
    q = np.broadcast_arrays(*q)
    outside = np.sqrt(sum(np.maximum(a, 0.0) ** 2 for a in q))
    inside = np.minimum(np.maximum(np.maximum(q[0], q[1]), q[2]), 0.0)
    return outside + inside
