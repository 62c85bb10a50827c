"""One time step of the coupled solver (Sec. 4.2, full time-stepping scheme).

Oracle (test infrastructure only).

For cycles k = 0 .. n_cycles-1 (the paper uses n_cycles = 2):
  1. advect phi with u^{n+1/2,k}; rebuild psi from the markers' centre of
     mass; cell and edge viscosity mu^{n+1,k+1} from (phi, psi)^{n+1,k+1};
  2. SSP-RK3 face density rho^{n+1,k+1} and the consistent convective term C
     from rho^n (level sets at t^n averaged onto faces);
     right-hand side  b = rho^n u^n/dt - C + (1-theta) L_mu^n u^n + rho_g g
     with rho_g = rho^flow(phi^{n+1,k+1}) on faces (well-balanced gravity,
     Sec. 5, for fully prescribed bodies) or rho^{n+1,k+1} (full gravity);
     solve  rho^{n+1,k+1}/dt u~ - theta L_mu u~ + G p = b,  -D u~ = 0;
  3. rigidity projection at X^{n+1/2,k} and the position update.
At k = 0: u^{n+1,0} = u^n, X^{n+1,0} = X^n.  At n = 0: u^{-1} = u^0.
With wave zones, u^{n+1} and phi^{n+1} are relaxed at t^{n+1} (Sec. 7.1).
With a Dirichlet inlet (waves.Inlet, Sec. 7.1) the x- faces hold the inlet's
normal velocity at the time of each velocity field; the implicit solve takes
the data at t^{n+1} (solve.solve_stokes_inlet), the explicit viscous term the
tangential data at t^n, and the transport's stage velocities the same
combinations of the data at t^n, t^{n-1}, t^{n+1} as of the velocities.
limiter selects the level-set face values ("cui" or "xsppm7", levelset.py).
With reinit_iters > 0, phi^{n+1} is then reinitialised to a signed distance
(Sec. 4.1; reinit.py) before the step is committed.

form = "nonconservative" takes the paper's non-conservative, inconsistent
formulation (Sec. 4.2.3) instead of step 2: the face density of the
momentum equation is rho^{n+1,k+1} from the level sets (no mass transport),
and the convection is the explicit CUI-limited N = div(u^{n+1/2,k} u^{n+1/2,k})
with u^{n+1/2,k} = (u^{n+1,k} + u^n)/2:
  rho^{n+1,k+1} (u~ - u^n)/dt + rho^{n+1,k+1} N = -G p + L_mu u (Crank-Nicolson
  split as above) + rho_g g.
Parity of this form is pinned in part (at rest; equal to the consistent form
for one density and a steady solenoidal flow); parity unpinned for the choice
of rho^{n+1,k+1} rather than rho^n in its mass term, which those cases cannot
separate.
"""
import numpy as np

from . import levelset, reinit, rigid, transport
from .grid import Grid
from .materials import Materials, face_average, flow_only
from .operators import strain_rate_apply
from .solve import solve_stokes, solve_stokes_inlet


class Props:
    def __init__(self, rho_l=1000.0, rho_g=1.2, rho_s=1000.0, mu_l=1e-3, mu_g=1.8e-5, mu_s=None,
                 n_cells=2.0, gravity=(0.0, 0.0, -9.81), gravity_mode="flow", theta=0.5):
        self.rho_l, self.rho_g, self.rho_s = rho_l, rho_g, rho_s
        self.mu_l, self.mu_g = mu_l, mu_g
        self.mu_s = max(mu_l, mu_g) if mu_s is None else mu_s
        self.n_cells = n_cells
        self.gravity = np.asarray(gravity, dtype=np.float64)
        self.gravity_mode = gravity_mode
        self.theta = theta


class Body:
    def __init__(self, X, dV, lock, U_pres=(0, 0, 0), W_pres=(0, 0, 0), half=None, cylinder=None):
        self.X = np.array(X, dtype=np.float64)
        self.dV = float(dV)
        self.lock = np.asarray(lock, dtype=bool)
        self.U_pres = np.asarray(U_pres, dtype=np.float64)
        self.W_pres = np.asarray(W_pres, dtype=np.float64)
        self.half = None if half is None else np.asarray(half, dtype=np.float64)
        # (radius, half length) of a cylinder along y, or None
        self.cylinder = None if cylinder is None else (float(cylinder[0]), float(cylinder[1]))
        self.Ub = np.zeros_like(self.X)
        self.Xcom = self.X.mean(axis=0)


class State:
    def __init__(self, g: Grid, props: Props, phi, psi, body=None, vel=None, p=None, zones=None, time=0.0,
                 inlet=None):
        self.g = g
        self.zones = zones  # waves.Zones or None (Sec. 7.1 relaxation at step end)
        self.inlet = inlet  # waves.Inlet or None (Sec. 7.1 Dirichlet inlet on the x- plane)
        self.time = time
        self.props = props
        self.phi = np.array(phi, dtype=np.float64)
        self.psi = np.array(psi, dtype=np.float64)
        self.body = body
        self.vel = [np.zeros(g.face_shape(c)) for c in range(3)] if vel is None else [np.array(a) for a in vel]
        self.gw = None
        if inlet is not None:
            self.vel[0][..., 0] = inlet.normal(g, time, props.n_cells)
            self.gw = inlet.tangential(g, time, props.n_cells)  # tangential data of vel
        self.vel_old = [a.copy() for a in self.vel]
        self.gw_old = None if self.gw is None else self.gw.copy()
        self.p = np.zeros(g.cell_shape) if p is None else np.array(p)


def _materials(s: State, phi, psi):
    pr = s.props
    return Materials(s.g, phi, psi, pr.rho_l, pr.rho_g, pr.rho_s, pr.mu_l, pr.mu_g, pr.mu_s, pr.n_cells)


def step(s: State, dt, n_cycles=2, reinit_iters=0, form="consistent", limiter="cui"):
    g, pr = s.g, s.props
    u_n = [a.copy() for a in s.vel]
    u_nm1 = [a.copy() for a in s.vel_old]
    phi_n, psi_n = s.phi.copy(), s.psi.copy()
    mat_n = _materials(s, phi_n, psi_n)
    rho_n = mat_n.rho_face
    inl = s.inlet
    gw_n = gw_nm1 = gw_np1 = gn_np1 = None
    if inl is not None:
        gw_n, gw_nm1 = s.gw, s.gw_old
        gw_np1 = inl.tangential(g, s.time + dt, pr.n_cells)
        gn_np1 = inl.normal(g, s.time + dt, pr.n_cells)
    Lmu_n = strain_rate_apply(g, mat_n, *u_n, inlet_w=gw_n)
    body = s.body
    X_n = body.X.copy() if body is not None else None
    Ub_n = body.Ub.copy() if body is not None else None
    u_k = [a.copy() for a in u_n]
    phi_k = phi_n.copy()
    X_k = X_n.copy() if body is not None else None
    psi_k = psi_n.copy()
    p = s.p.copy()
    info = {}
    for k in range(n_cycles):
        u_half = [0.5 * (a + b) for a, b in zip(u_k, u_n)]
        phi_new = levelset.advect(g, u_half, phi_n, 0.5 * (phi_k + phi_n), dt, limiter=limiter)
        if body is not None and body.half is not None:
            psi_new = levelset.box_sdf(g, X_k.mean(axis=0), body.half)
        elif body is not None and body.cylinder is not None:
            psi_new = levelset.cylinder_sdf(g, X_k.mean(axis=0), *body.cylinder)
        else:
            psi_new = psi_k
        mat = _materials(s, phi_new, psi_new)
        gw_k = gw_n if k == 0 else gw_np1  # tangential inlet data of u_k
        if form == "consistent":
            u1, u2 = transport.rk_velocities(u_n, u_nm1, u_k, k)
            g2 = None if inl is None else transport.rk_velocities([gw_n], [gw_nm1], [gw_k], k)[1][0]
            rho_new, C = transport.ssp_rk3(g, rho_n, u_n, u1, u2, dt, inlet_w2=g2)
        elif form == "nonconservative":
            rho_new = mat.rho_face
            ones = [np.ones(g.face_shape(c)) for c in range(3)]
            N = transport.convective(g, [0.5 * (a + b) for a, b in zip(u_k, u_n)], ones,
                                     None if inl is None else 0.5 * (gw_k + gw_n))
        else:
            raise ValueError(form)
        if pr.gravity_mode == "flow":
            rho_grav = [flow_only(face_average(g, phi_new, c), pr.rho_l, pr.rho_g, mat.eps) for c in range(3)]
        else:
            rho_grav = rho_new
        if form == "consistent":
            b_u = [rho_n[c] * u_n[c] / dt - C[c] + (1.0 - pr.theta) * Lmu_n[c] + rho_grav[c] * pr.gravity[c]
                   for c in range(3)]
        else:
            b_u = [rho_new[c] * (u_n[c] / dt - N[c]) + (1.0 - pr.theta) * Lmu_n[c] + rho_grav[c] * pr.gravity[c]
                   for c in range(3)]
        b = g.pack(b_u[0], b_u[1], b_u[2], np.zeros(g.cell_shape))
        if inl is None:
            x = solve_stokes(g, mat, rho_new, dt, pr.theta, b)
        else:
            x = solve_stokes_inlet(g, mat, rho_new, dt, pr.theta, b, gn_np1, gw_np1)
        ut, vt, wt, p = g.unpack(x)
        vel_t = [ut, vt, wt]
        if body is not None:
            X_half = 0.5 * (X_k + X_n)
            vel_c, Ub, Ur, Wr, Xc, Ui = rigid.constrain(g, vel_t, X_half, body.dV, body.lock,
                                                        body.U_pres, body.W_pres, full=True)
            X_k = rigid.update_positions(X_n, Ub, Ub_n, dt)
            info.update(Ur=Ur, Wr=Wr, Ub=Ub,
                        F_lm=rigid.lm_force(Ub, Ub_n, Ub - Ui, pr.rho_s, body.dV, dt))
        else:
            vel_c = vel_t
        u_k = vel_c
        phi_k = phi_new
        psi_k = psi_new
        info.setdefault("u_tilde", []).append(vel_t)
    if s.zones is not None:
        u_k, phi_k = s.zones.relax(g, u_k, phi_k, s.time + dt, pr.n_cells)
    if reinit_iters > 0:
        phi_k = reinit.reinit(g, phi_k, reinit_iters)
    s.time += dt
    s.vel_old = u_n
    s.vel = u_k
    if inl is not None:
        s.gw_old, s.gw = gw_n, gw_np1
    s.p = p
    s.phi = phi_k
    s.psi = psi_k
    if body is not None:
        body.X = X_k
        body.Ub = info["Ub"]
        body.Xcom = X_k.mean(axis=0)
    return info
