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
