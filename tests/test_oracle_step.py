"""Pins for the oracle's full time step (Sec. 4.2): the hydrostatic
three-phase tank with a locked body keeps zero velocity to round-off over
several steps with the well-balanced gravity of Sec. 5, and develops
spurious currents with the full rho g (the contrast of Sec. 8.4)."""
import numpy as np

from oracle.grid import Grid
from oracle import step as st
from paper_1901_07892_gb300 import inputs


def _run(mode, nsteps):
    c = inputs.tank3d(n=10, with_body=True, dt=5e-4, gravity_mode=mode)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    pr = st.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l if mode == "flow" else c.rho_s,
                  mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity, gravity_mode=mode)
    body = st.Body(c.markers, c.dV, [True] * 6, half=c.box_half)
    s = st.State(g, pr, c.phi, c.psi, body)
    for _ in range(nsteps):
        st.step(s, c.dt)
    return max(np.abs(a).max() for a in s.vel), s


def test_hydrostatic_tank_stays_at_rest():
    umax, s = _run("flow", 3)
    assert umax < 1e-12
    # the pressure is hydrostatic: p varies only with z
    p = s.p
    assert np.abs(p - p[:, :1, :1]).max() < 1e-8 * np.abs(p).max()


def test_full_gravity_drives_spurious_currents():
    umax, _ = _run("full", 1)
    assert umax > 1e-6


def test_nonconservative_hydrostatic_tank_stays_at_rest():
    """The non-conservative form (Sec. 4.2.3) from rest: N = 0 and the
    level-set density times u^n/dt vanish, so the well-balanced gravity keeps
    the tank at rest exactly as in the consistent form."""
    c = inputs.tank3d(n=10, with_body=True, dt=5e-4, gravity_mode="flow")
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    pr = st.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                  gravity_mode="flow")
    s = st.State(g, pr, c.phi, c.psi, st.Body(c.markers, c.dV, [True] * 6, half=c.box_half))
    for _ in range(2):
        st.step(s, c.dt, form="nonconservative")
    assert max(np.abs(a).max() for a in s.vel) < 1e-12


def _stream_velocity(g, amp=0.3):
    """A discretely divergence-free MAC velocity with zero normal velocity on
    the walls: u = d psi/dy, v = -d psi/dx of a node stream function that
    vanishes on the boundary, w = 0, the same in every z-plane."""
    X, Y = np.meshgrid(np.arange(g.nx + 1) * g.hx, np.arange(g.ny + 1) * g.hy, indexing="xy")
    psi = amp * np.sin(np.pi * X / g.lx) ** 2 * np.sin(np.pi * Y / g.ly) ** 2 * (1 + X * Y)
    u = (psi[1:, :] - psi[:-1, :]) / g.hy          # (ny, nx+1)
    v = -(psi[:, 1:] - psi[:, :-1]) / g.hx         # (ny+1, nx)
    return [np.broadcast_to(u, g.face_shape(0)).copy(), np.broadcast_to(v, g.face_shape(1)).copy(),
            np.zeros(g.face_shape(2))]


def test_forms_agree_for_uniform_density_and_steady_solenoidal_flow():
    """One cycle of the first step with a single density and a divergence-free
    u^0 = u^{-1}: the SSP-RK3 transport keeps the face density constant and
    its velocities u^(1), u^(2) equal u^0, which is also u^{n+1/2,0}; the
    consistent C is then rho N and the two forms solve the same system.  A
    dropped density factor or a wrong sign of N in the non-conservative
    right-hand side breaks the agreement."""
    g = Grid(12, 10, 6, 1.0, 0.9, 0.6, (-1.0, -1.0, -1.0, -1.0, 1.0, 1.0))
    vel = _stream_velocity(g)
    x = (np.arange(g.nx) + 0.5) * g.hx
    div = sum(np.diff(vel[d], axis=2 - d) / g.h[d] for d in range(3))
    assert np.abs(div).max() < 1e-13
    pr = st.Props(rho_l=1000.0, rho_g=1000.0, rho_s=1000.0, mu_l=1e-3, mu_g=1e-3, mu_s=1e-3,
                  gravity=(0.0, 0.0, -9.81), gravity_mode="full")
    phi = np.broadcast_to(x - 0.45, g.cell_shape).copy()
    out = {}
    for form in ("consistent", "nonconservative"):
        s = st.State(g, pr, phi, np.ones(g.cell_shape), None, vel=vel)
        st.step(s, 2e-3, n_cycles=1, form=form)
        out[form] = np.concatenate([a.ravel() for a in s.vel])
    ref = out["consistent"]
    assert np.abs(ref - np.concatenate([a.ravel() for a in vel])).max() > 1e-6  # the flow did change
    assert np.abs(out["nonconservative"] - ref).max() < 1e-10 * np.abs(ref).max()


def test_forms_differ_at_high_density_ratio():
    """With air and water and a moving interface the forms are different
    schemes (the inconsistency of Sec. 4.2.3): two steps from a wavy surface
    leave velocities that differ well above round-off."""
    c = inputs.tank3d(n=8, seed=3, with_body=False, dt=2e-3, gravity_mode="full")
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    pr = st.Props(rho_l=c.rho_l, rho_g=c.rho_g, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity, gravity_mode="full")
    out = {}
    for form in ("consistent", "nonconservative"):
        s = st.State(g, pr, c.phi, c.psi)
        for _ in range(2):
            st.step(s, c.dt, form=form)
        out[form] = np.concatenate([a.ravel() for a in s.vel])
    assert np.abs(out["consistent"] - out["nonconservative"]).max() > 1e-6 * np.abs(out["consistent"]).max()


def test_two_dimensional_hydrostatic_step():
    """A 2-D tank (nz = 1, free-slip z walls: every z-derivative vanishes and
    the w-faces are all wall faces) with a locked square at rest stays at
    rest in both formulations."""
    n = 16
    c = inputs.tank2d(n=n, with_body=True)
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    pr = st.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                  gravity_mode="flow")
    for form in ("consistent", "nonconservative"):
        s = st.State(g, pr, c.phi, c.psi, st.Body(c.markers, c.dV, [True] * 6, half=c.box_half))
        for _ in range(2):
            st.step(s, c.dt, form=form)
        assert max(np.abs(a).max() for a in s.vel) < 1e-12, form
