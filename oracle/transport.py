"""Consistent mass/momentum transport on face-centred control volumes
(Sec. 4.2.2, conservative and consistent formulation).

Oracle (test infrastructure only).

Face density is integrated with SSP-RK3 (the three stage equations of
Sec. 4.2.2); the convective term C reuses the stage-3 advective velocity and
limited density, multiplied by the limited velocity, which couples mass and
momentum transport.

Readings (the paper defers these details to its reference on the
consistent scheme):
* The control volume of a c-face spans from the cell centre on one side to
  the cell centre on the other along c, and between edges across c.
  Its faces along c sit at cell centres, where the advective velocity is the
  mean of the two c-faces; its faces along d != c sit on edges, where the
  advective velocity is the mean of the two d-faces adjacent along c.
* Limited values come from the cubic-upwind interpolation (CUI, kappa = 1/3)
  bounded by the convection-boundedness criterion in normalized variables:
      t = (q_C - q_U)/(q_D - q_U)
      t_f = 3t (0 < t <= 2/13), 5t/6 + 1/3 (2/13 < t <= 4/5), 1 (4/5 < t <= 1),
      t otherwise;   q_f = q_U + t_f (q_D - q_U)   (q_f = q_C when q_D = q_U).
  C is the upwind point, U the next point upwind, D the downwind point; the
  direction comes from the sign of the advective velocity (> 0: from below).
* Ghosts: face density mirrors evenly across walls (Neumann); velocity
  ghosts follow the wall condition (tangential: sign s, normal: odd; across
  an open top the normal velocity mirrors evenly, its derivative being zero
  there, grid.py).
* Faces on walls are not transported (R = C = 0 there).
* Across a Dirichlet inlet (Sec. 7.1) the ghosts of the tangential w are
  2 w_b - (mirror image), with w_b the inlet data of the velocity being
  transported; a stage velocity's data are the same combination of the data
  at t^n, t^{n-1} and t^{n+1} as the stage velocity itself.
"""
import numpy as np

from .grid import Grid


def cui(qU, qC, qD):
    den = qD - qU
    safe = np.where(den == 0.0, 1.0, den)
    t = (qC - qU) / safe
    tf = np.where((t > 0.0) & (t <= 2.0 / 13.0), 3.0 * t,
         np.where((t > 2.0 / 13.0) & (t <= 0.8), 5.0 * t / 6.0 + 1.0 / 3.0,
         np.where((t > 0.8) & (t <= 1.0), 1.0, t)))
    return np.where(den == 0.0, qC, qU + tf * den)


def _ghost_extend(g: Grid, q, c, d, kind, lo_data=None):
    """Extend array q (values on c-faces, or on cells if c is None) by two
    ghost layers on both ends of axis d.
    kind: 'even' (density / scalars), 'vel' (velocity component c).
    lo_data: Dirichlet data of a tangential velocity on the lower plane of
    axis d (the inlet's w): its ghosts are 2 data - (mirror image)."""
    ax = q.ndim - 1 - d
    n = q.shape[ax]
    face_along_d = (c == d)
    idx_lo = []
    idx_hi = []
    sgn_lo = []
    sgn_hi = []
    for gl in (2, 1):  # ghost layer distances, outermost first
        if face_along_d:
            # stored 0..n-1 (n = cells+1); wall faces at 0 and n-1
            idx_lo.append(gl)
            idx_hi.append(n - 1 - gl)
        else:
            idx_lo.append(gl - 1)
            idx_hi.append(n - gl)
        if kind == "even":
            sgn_lo.append(1.0)
            sgn_hi.append(1.0)
        elif face_along_d:
            sgn_lo.append(-1.0)
            sgn_hi.append(1.0 if (d == 2 and g.open_top) else -1.0)
        else:
            sgn_lo.append(g.sign(d, 0))
            sgn_hi.append(g.sign(d, 1))
    idx_lo = [min(max(i, 0), n - 1) for i in idx_lo]
    idx_hi = [min(max(i, 0), n - 1) for i in idx_hi]
    lo = [np.take(q, [i], axis=ax) * s for i, s in zip(idx_lo, sgn_lo)]
    if lo_data is not None:
        lo = [a + 2.0 * np.expand_dims(lo_data, ax) for a in lo]
    hi = [np.take(q, [i], axis=ax) * s for i, s in zip(idx_hi[::-1], sgn_hi[::-1])]
    return np.concatenate(lo + [q] + hi, axis=ax)


def _limited(g: Grid, q, c, d, adv, kind, on_cells, lo_data=None):
    """Limited value of q (a c-face array, extended along d) at the CV faces
    along d.  on_cells: CV faces along d are between consecutive q entries
    m and m+1 (d == c), indexed m = 0..n-2; otherwise between m-1 and m,
    m = 0..n (edges, the two ends on walls)."""
    e = _ghost_extend(g, q, c, d, kind, lo_data)
    ax = e.ndim - 1 - d
    n = q.shape[q.ndim - 1 - d]

    def take(off, count):
        return np.take(e, np.arange(off, off + count), axis=ax)

    if on_cells:
        cnt = n - 1
        # lower point m -> extended index m+2
        qm1, q0, q1, q2 = take(1, cnt), take(2, cnt), take(3, cnt), take(4, cnt)
    else:
        cnt = n + 1
        # CV face m between q[m-1] and q[m]; q[m-1] -> extended m+1
        qm1, q0, q1, q2 = take(0, cnt), take(1, cnt), take(2, cnt), take(3, cnt)
    pos = cui(qm1, q0, q1)
    neg = cui(q2, q1, q0)
    return np.where(adv > 0.0, pos, neg)


def _adv_velocity(g: Grid, vel, c, d):
    """Advective velocity on the CV faces of c-faces along direction d."""
    if d == c:
        q = vel[c]
        ax = q.ndim - 1 - d
        n = q.shape[ax]
        return 0.5 * (np.take(q, np.arange(0, n - 1), axis=ax) + np.take(q, np.arange(1, n), axis=ax))
    q = vel[d]  # d-faces; average the two adjacent along c
    axc = q.ndim - 1 - c
    n = q.shape[axc]
    a = 0.5 * (np.take(q, np.arange(0, n - 1), axis=axc) + np.take(q, np.arange(1, n), axis=axc))
    # a lives at the c-face positions interior along c: pad the two wall
    # positions along c with zeros (those c-faces are not transported; with
    # one cell along c, as for w in 2-D, there are no interior positions)
    shape = list(a.shape)
    shape[axc] = 1
    z = np.zeros(shape)
    return np.concatenate([z, a, z], axis=axc)


def _fluxes(g: Grid, vel, rho, qvel, c, inlet_w=None):
    """Divergence over the c-face control volumes of adv * rho_lim (* q_lim);
    inlet_w: tangential inlet data of qvel = w on the x- plane, or None."""
    out = np.zeros(g.face_shape(c))
    for d in range(3):
        adv = _adv_velocity(g, vel, c, d)
        on_cells = d == c
        r_lim = _limited(g, rho, c, d, adv, "even", on_cells)
        F = adv * r_lim
        if qvel is not None:
            data = inlet_w if (c == 2 and d == 0) else None
            F = F * _limited(g, qvel, c, d, adv, "vel", on_cells, data)
        ax = F.ndim - 1 - d
        n = F.shape[ax]
        dF = (np.take(F, np.arange(1, n), axis=ax) - np.take(F, np.arange(0, n - 1), axis=ax)) / g.h[d]
        if on_cells:
            # c-face m (interior 1..n-1) has CV faces at cells m-1 and m
            axc = out.ndim - 1 - c
            idx = [slice(None)] * out.ndim
            idx[axc] = slice(1, -1)
            out[tuple(idx)] += dF
        else:
            out += dF
    ax = out.ndim - 1 - c
    idx = [slice(None)] * out.ndim
    idx[ax] = 0
    out[tuple(idx)] = 0.0
    idx[ax] = -1
    out[tuple(idx)] = 0.0
    return out


def mass_flux(g: Grid, vel, rho):
    """R(u_adv, rho_lim) for the three face-density arrays."""
    return [_fluxes(g, vel, rho[c], None, c) for c in range(3)]


def convective(g: Grid, vel, rho, inlet_w=None):
    """C(u_adv, rho_lim u_lim) for the three momentum components; inlet_w:
    the tangential inlet data of vel's w, or None."""
    return [_fluxes(g, vel, rho[c], vel[c], c, inlet_w) for c in range(3)]


def rk_velocities(u_n, u_nm1, u_k, k):
    """u^(1), u^(2) of Sec. 4.2.2 for cycle k."""
    if k == 0:
        u1 = [2.0 * a - b for a, b in zip(u_n, u_nm1)]
        u2 = [1.5 * a - 0.5 * b for a, b in zip(u_n, u_nm1)]
    else:
        u1 = [a for a in u_k]
        u2 = [0.375 * a + 0.75 * b - 0.125 * c for a, b, c in zip(u_k, u_n, u_nm1)]
    return u1, u2


def ssp_rk3(g: Grid, rho_n, u_n, u1, u2, dt, inlet_w2=None):
    """Returns rho^{n+1,k+1} (3 face arrays) and C (3 face arrays);
    inlet_w2: the tangential inlet data of u2's w, or None."""
    R0 = mass_flux(g, u_n, rho_n)
    r1 = [rho_n[c] - dt * R0[c] for c in range(3)]
    R1 = mass_flux(g, u1, r1)
    r2 = [0.75 * rho_n[c] + 0.25 * r1[c] - 0.25 * dt * R1[c] for c in range(3)]
    R2 = mass_flux(g, u2, r2)
    r3 = [rho_n[c] / 3.0 + 2.0 / 3.0 * r2[c] - 2.0 / 3.0 * dt * R2[c] for c in range(3)]
    C = convective(g, u2, r2, inlet_w2)
    return r3, C
