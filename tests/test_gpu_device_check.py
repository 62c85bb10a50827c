"""The device bound check of the marker update: a locked box driven at a
prescribed velocity towards the x = 1 wall steps normally while its markers
are inside the box and reports WSI_ERR_DEVICE on the step that carries one
beyond the wall by more than half a cell (the interpolation and spreading
taps reflect and zero any tap outside the grid, so such a marker reads and
writes in-bounds cells only).  The flag is cleared: the context stays
usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1901_07892_gb300 import inputs, wsi


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def test_marker_leaving_the_box_sets_device_flag():
    c = inputs.tank3d(n=16, seed=None, with_body=True)
    h = 1.0 / 16
    U, dt = 2.0, 0.01  # CFL U dt / h = 0.32
    ctx = wsi.Context.from_case(c, precision=wsi.PREC_MIXED)
    ctx.set_case(c, U_pres=(U, 0.0, 0.0))
    xmax = float(np.max(c.markers[:, 0]))
    # the previous body velocity starts at zero, so after k steps the markers
    # have moved U dt (k - 1/2); k_out is the first step past 1 + h/2
    k_out = int(np.floor((1.0 + 0.5 * h - xmax) / (U * dt) + 0.5)) + 1
    assert 1 < k_out < 40
    for k in range(1, k_out):
        ctx.step(dt, rtol=1e-8)
        assert xmax + (k - 0.5) * U * dt <= 1.0 + 0.5 * h
    with pytest.raises(wsi.WsiError) as e:
        ctx.step(dt, rtol=1e-8)
    assert e.value.code == wsi.ERR_DEVICE, e.value
    assert "marker" in str(e.value)
    # flag cleared; the fields of the committed step are readable and finite
    p = ctx.get_field(wsi.F_P)
    assert np.all(np.isfinite(np.asarray(p)))
    ctx.close()
