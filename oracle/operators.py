"""Second-order staggered-grid operators (Sec. 3.1) and the implicit Stokes
operator of the conservative momentum equation (Sec. 4.2.2).

Oracle (test infrastructure only).  Matrix-free numpy; every function
accepts leading batch axes on its field arguments.

  G p        pressure gradient on faces           (p_i - p_{i-1})/h
  D u        divergence at cell centres           sum_d (u_{i+1} - u_i)/h_d
  L_beta p = D (beta G p),  beta = 1/rho on faces (the pressure operator)
  L_mu u   = div_h[ mu (grad_h u + grad_h u^T) ]    (strain-rate operator)
  A u      = rho/dt u - theta L_mu u                 (implicit viscous block;
             theta = 1/2 is the paper's Crank-Nicolson weight, Sec. 4.2.2)
  K [u;p]  = [A u + G p ; -D u]                       (Stokes saddle operator)

Normal stress uses mu at cell centres; shear stress uses the harmonically
averaged mu on edges.  Faces on walls are not unknowns: every face-valued
result is 0 there.  With an open top (grid.py) the top w-faces are rows too:
G p there is (0 - p)/(h/2) from the pressure ghost -p; the normal stress of
the ghost cell above is minus that of the cell below (w[nz+1] = w[nz-1]); the
shear stresses on the top edges take the tangential ghosts -u, -v.

Dirichlet inlet (Sec. 7.1) on the x- side: its faces are not unknowns but
hold the prescribed normal velocity, which every operator reads like any
other entry of u; the prescribed tangential velocity w_b of the x- edges
(inlet_w, shape (nz+1, ny)) enters through the ghost of w across the plane,
2 w_b - w (zero-data: the no-slip ghost -w).  The inlet's span-wise
velocity is zero (the no-slip ghost).
"""
import numpy as np

from .grid import Grid, pad_tangential


def _zero_wall_faces(g: Grid, r, c):
    ax = r.ndim - 1 - c
    idx = [slice(None)] * r.ndim
    idx[ax] = 0
    r[tuple(idx)] = 0.0
    if not (c == 2 and g.open_top):
        idx[ax] = -1
        r[tuple(idx)] = 0.0
    return r


def _diff(a, axis_from_end, h):
    """Forward difference along an axis counted from the end (0 = x)."""
    ax = a.ndim - 1 - axis_from_end
    n = a.shape[ax]
    return (np.take(a, np.arange(1, n), axis=ax) - np.take(a, np.arange(0, n - 1), axis=ax)) / h


def grad(g: Grid, p):
    """G p on u, v, w faces; zero on wall faces."""
    out = []
    for c in range(3):
        hc = g.h[c]
        ax = p.ndim - 1 - c
        d = _diff(p, c, hc)
        shp = list(p.shape)
        shp[ax] += 1
        r = np.zeros(shp)
        idx = [slice(None)] * p.ndim
        idx[ax] = slice(1, -1)
        r[tuple(idx)] = d
        if c == 2 and g.open_top:
            idx[ax] = -1
            r[tuple(idx)] = -2.0 * np.take(p, -1, axis=ax) / hc
        out.append(r)
    return out


def div(g: Grid, u, v, w):
    """D u at cell centres."""
    return _diff(u, 0, g.hx) + _diff(v, 1, g.hy) + _diff(w, 2, g.hz)


def pressure_apply(g: Grid, beta, p):
    """L_beta p = D(beta G p); beta = (beta_x, beta_y, beta_z) on faces."""
    gp = grad(g, p)
    return div(g, beta[0] * gp[0], beta[1] * gp[1], beta[2] * gp[2])


def strain_rate_apply(g: Grid, mat, u, v, w, inlet_w=None):
    """L_mu u = div_h[mu (grad_h u + grad_h u^T)] for all three components,
    evaluated on every face (wall faces set to 0); inlet_w: tangential
    inlet data on the x- edges, or None."""
    hx, hy, hz = g.h
    vel = (u, v, w)
    mu_edge = {(0, 1): mat.mu_xy, (0, 2): mat.mu_xz, (1, 2): mat.mu_yz}
    mu_cc = mat.mu_cc
    out = []
    for c in range(3):
        q = vel[c]
        top = c == 2 and g.open_top  # the last c-face is a row too
        end = None if top else -1
        # normal stress 2 mu dq/dx_c at cells, differenced back onto faces
        dq = _diff(q, c, g.h[c])                      # at cells
        tau = 2.0 * mu_cc * dq
        ax = q.ndim - 1 - c
        if top:
            # ghost cell above the open top: minus the stress of the cell below
            tau = np.concatenate([tau, -np.take(tau, [-1], axis=ax)], axis=ax)
        res = np.zeros(q.shape)
        idx = [slice(None)] * q.ndim
        idx[ax] = slice(1, end)
        res[tuple(idx)] = _diff(tau, c, g.h[c])
        # shear stresses on edges in the (c, d) planes
        qp = pad_tangential(g, q, c)
        if c == 2 and inlet_w is not None:
            qp = qp.copy()
            qp[..., 1:-1, 0] += 2.0 * inlet_w  # ghost 2 w_b - w across the inlet
        for d in range(3):
            if d == c:
                continue
            key = (min(c, d), max(c, d))
            mu_e = mu_edge[key]
            # dq/dx_d on the (c,d) edges: difference of padded q along d
            dqd = _diff(qp, d, g.h[d])
            # strip the padding along the third axis e
            e = 3 - c - d
            axe = dqd.ndim - 1 - e
            ne = dqd.shape[axe]
            dqd = np.take(dqd, np.arange(1, ne - 1), axis=axe)
            # d-component differenced along c: defined on edges interior in c
            # (and on the open top's edges, across the tangential ghost)
            vd = vel[d]
            if top:
                vd = np.concatenate([vd, g.sign(c, 1) * np.take(vd, [-1], axis=vd.ndim - 1 - c)],
                                    axis=vd.ndim - 1 - c)
            dv = _diff(vd, c, g.h[c])
            # dqd has full extent along c (q is a c-face array); dv lacks the
            # wall positions along c.  Shear flux only needed at c-face rows.
            axc = dqd.ndim - 1 - c
            nc = dqd.shape[axc]
            last = nc if top else nc - 1
            dqd_int = np.take(dqd, np.arange(1, last), axis=axc)
            axm = mu_e.ndim - 1 - c
            mu_int = np.take(mu_e, np.arange(1, mu_e.shape[axm] if top else mu_e.shape[axm] - 1), axis=axm)
            flux = mu_int * (dqd_int + dv)
            sh = _diff(flux, d, g.h[d])
            res[tuple(idx)] += sh
        out.append(_zero_wall_faces(g, res, c))
    return out


def viscous_apply(g: Grid, mat, rho_face, dt, theta, u, v, w, inlet_w=None):
    """A u = rho/dt u - theta L_mu u (wall faces 0)."""
    L = strain_rate_apply(g, mat, u, v, w, inlet_w)
    out = []
    for c, q in enumerate((u, v, w)):
        r = rho_face[c] / dt * q - theta * L[c]
        out.append(_zero_wall_faces(g, r, c))
    return out


def stokes_apply(g: Grid, mat, rho_face, dt, theta, x, inlet_w=None):
    """K x for a packed Stokes vector x = (u, v, w, p); with inlet_w the
    affine operator of the Dirichlet inlet (its data: x's x- faces and
    inlet_w)."""
    u, v, w, p = g.unpack(x)
    au = viscous_apply(g, mat, rho_face, dt, theta, u, v, w, inlet_w)
    gp = grad(g, p)
    ru = [_zero_wall_faces(g, au[c] + gp[c], c) for c in range(3)]
    rp = -div(g, u, v, w)
    return g.pack(ru[0], ru[1], ru[2], rp)
