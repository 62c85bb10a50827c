"""Parity of the non-conservative, inconsistent formulation (Sec. 4.2.3)
with the oracle's step: two full time steps of a 3-D tank with a wavy
surface and a locked box, in both precisions, solved to 1e-13 so that the
field tolerance of the consistent step tests applies."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import step as ost
from oracle.grid import Grid
from paper_1901_07892_gb300 import inputs, wsi

FIELD_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("precision", [wsi.PREC_FP64, wsi.PREC_MIXED])
@pytest.mark.parametrize("gravity_mode", ["flow", "full"])
def test_nonconservative_step_parity(precision, gravity_mode):
    c = inputs.tank3d(nxyz=(20, 16, 8), seed=11, dt=5e-4, gravity_mode=gravity_mode)
    c.rho_s = c.rho_l
    g = Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, c.bc)
    ctx = wsi.Context.from_case(c, precision=precision, restart=30, transport_form=wsi.FORM_NONCONSERVATIVE)
    ctx.set_case(c, rho_s=c.rho_l)
    pr = ost.Props(rho_l=c.rho_l, rho_g=c.rho_g, rho_s=c.rho_l, mu_l=c.mu_l, mu_g=c.mu_g, gravity=c.gravity,
                   gravity_mode=gravity_mode)
    s = ost.State(g, pr, c.phi, c.psi, ost.Body(c.markers, c.dV, [True] * 6, half=c.box_half))
    for _ in range(2):
        ctx.step(c.dt, rtol=1e-13, max_iters=600)
        ost.step(s, c.dt, form="nonconservative")
    vel = np.asarray(ctx.get_field(wsi.F_VEL))
    ref = np.concatenate([a.ravel() for a in s.vel])
    print(precision, gravity_mode, "vel", _rel(vel, ref))
    assert _rel(vel, ref) < FIELD_TOL
    p = np.asarray(ctx.get_field(wsi.F_P))
    assert _rel(p - p.mean(), (s.p - s.p.mean()).ravel()) < FIELD_TOL
    assert _rel(np.asarray(ctx.get_field(wsi.F_PHI)), s.phi.ravel()) < 1e-9
    ctx.close()


def test_unknown_form_is_refused():
    with pytest.raises(wsi.WsiError) as e:
        wsi.Context(8, 8, 8, transport_form=7)
    assert e.value.code == wsi.ERR_INVALID_ARG
