"""Level-set advection (Sec. 4.2.1) and the structure level set (Sec. 4.1).

Oracle (test infrastructure only).

  phi^{n+1,k+1} = phi^n - dt Q(u^{n+1/2,k}, phi^{n+1/2,k})

with Q the conservative flux divergence div(u phi) on cell centres and the
face values of phi taken upwind: either limited by the bounded cubic-upwind
(CUI) scheme of the momentum transport (the default stand-in), or by the
paper's xsPPM7 limiter, read as below (the paper names it and cites its
references without printing it).  Homogeneous Neumann ghosts for phi on
every wall; faces on walls carry zero velocity and hence zero flux.

The structure level set is rebuilt every cycle from the markers' centre of
mass as an analytic signed distance (Sec. 4.1): for a box of half-extents
a about centre X_c,  q = |x - X_c| - a,  psi = |max(q, 0)| + min(max_d q_d, 0).
"""
import numpy as np

from .grid import Grid
from .transport import cui


def _mirror(i, n):
    """Index of the even (Neumann) mirror image of cell i in 0..n-1."""
    for _ in range(8):
        if i < 0:
            i = -1 - i
        elif i >= n:
            i = 2 * n - 1 - i
    return min(max(i, 0), n - 1)


def _extend_even(q, d, layers=2):
    ax = q.ndim - 1 - d
    n = q.shape[ax]
    ids = [_mirror(i, n) for i in range(-layers, 0)] + list(range(n)) + \
          [_mirror(i, n) for i in range(n, n + layers)]
    return np.take(q, ids, axis=ax)


# ---------------------------------------------------------------------------
# xsPPM7 (Sec. 4.2.1 names the limiter and cites its references without
# printing it).  Reading: the upwind face value is the seventh-order
# upwind-biased interpolant of the seven nearest cell values (the values
# taken as cell averages), limited to the monotonicity-preserving bounds of
# Suresh and Huynh with their curvature terms (alpha = 4), which admit smooth
# extrema instead of clipping them.  Arguments are ordered along the flow:
# q0 is the upwind cell of the face, qp1 the downwind cell.

def minmod(a, b):
    return 0.5 * (np.sign(a) + np.sign(b)) * np.minimum(np.abs(a), np.abs(b))


def minmod4(a, b, c, d):
    s = np.sign(a)
    same = (np.sign(b) == s) & (np.sign(c) == s) & (np.sign(d) == s)
    return np.where(same, s * np.minimum(np.minimum(np.abs(a), np.abs(b)), np.minimum(np.abs(c), np.abs(d))), 0.0)


def interp7(qm3, qm2, qm1, q0, qp1, qp2, qp3):
    """Seventh-order face value between q0 and qp1 from the cell values
    q_{-3}..q_{+3} (exact for cell averages of polynomials of degree 6)."""
    return (-3.0 * qm3 + 25.0 * qm2 - 101.0 * qm1 + 319.0 * q0 + 214.0 * qp1 - 38.0 * qp2 + 4.0 * qp3) / 420.0


def xsppm7(qm3, qm2, qm1, q0, qp1, qp2, qp3, alpha=4.0):
    u7 = interp7(qm3, qm2, qm1, q0, qp1, qp2, qp3)
    ump = q0 + minmod(qp1 - q0, alpha * (q0 - qm1))
    dm1 = qm2 - 2.0 * qm1 + q0
    d0 = qm1 - 2.0 * q0 + qp1
    dp1 = q0 - 2.0 * qp1 + qp2
    dp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1)    # curvature at the face
    dm = minmod4(4.0 * dm1 - d0, 4.0 * d0 - dm1, dm1, d0)    # curvature at the face upwind
    uul = q0 + alpha * (q0 - qm1)
    umd = 0.5 * (q0 + qp1) - 0.5 * dp
    ulc = q0 + 0.5 * (q0 - qm1) + 4.0 / 3.0 * dm
    umin = np.maximum(np.minimum(np.minimum(q0, qp1), umd), np.minimum(np.minimum(q0, uul), ulc))
    umax = np.minimum(np.maximum(np.maximum(q0, qp1), umd), np.maximum(np.maximum(q0, uul), ulc))
    limited = u7 + minmod(umin - u7, umax - u7)   # median(u7, umin, umax)
    return np.where((u7 - q0) * (u7 - ump) <= 0.0, u7, limited)


def advect(g: Grid, vel, phi_n, phi_half, dt, limiter="cui"):
    """limiter: "cui" (the stand-in: bounded cubic upwind) or "xsppm7"."""
    Q = np.zeros(g.cell_shape)
    layers = 2 if limiter == "cui" else 4
    for d in range(3):
        e = _extend_even(phi_half, d, layers)
        ax = e.ndim - 1 - d
        n = phi_half.shape[phi_half.ndim - 1 - d]
        cnt = n + 1  # faces 0..n; face m between cells m-1 and m

        def take(off):
            # cell m - 1 + off - (layers - 1) ... relative to face m: off = 0 is cell m - layers
            return np.take(e, np.arange(off, off + cnt), axis=ax)

        a = vel[d]
        if limiter == "cui":
            qm2, qm1, q0, q1 = take(0), take(1), take(2), take(3)
            lim = np.where(a > 0.0, cui(qm2, qm1, q0), cui(q1, q0, qm1))
        elif limiter == "xsppm7":
            # cells m-4 .. m+3 around face m
            c = [take(o) for o in range(8)]
            pos = xsppm7(c[0], c[1], c[2], c[3], c[4], c[5], c[6])
            neg = xsppm7(c[7], c[6], c[5], c[4], c[3], c[2], c[1])
            lim = np.where(a > 0.0, pos, neg)
        else:
            raise ValueError(limiter)
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
