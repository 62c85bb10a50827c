"""The allocation-free norm entry point against the library's own pressure
solve: the relative residual it reports equals ||y - L x|| / ||y|| formed
from the returned x with the existing operator entry point and the norms
taken by the allocation-free call, on two calls in a row (deterministic);
sizes beyond the static scratch are rejected.  Collected last on purpose:
it must pass after every other test as well as alone."""
import ctypes

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


def test_norm_matches_pressure_solve_residual_twice():
    c = inputs.tank3d(n=32, seed=5, with_body=False)
    ctx = wsi.Context.from_case(c, precision=wsi.PREC_FP64)
    ctx.set_case(c, with_body=False)
    y = torch.from_numpy(inputs.random_cells(c.phi.shape, 5).ravel()).cuda()
    y -= y.mean()
    x, st = wsi.pressure_solve(ctx, y.clone(), rtol=1e-6, max_cycles=50)
    r = y - ctx.apply(wsi.OP_PRESSURE, x)
    r -= r.mean()
    got = []
    for _ in range(2):
        rel = wsi.norm2_noalloc(r) / wsi.norm2_noalloc(y)
        assert rel == pytest.approx(st.rel_residual, rel=1e-9)
        got.append(rel)
    assert got[0] == got[1]
    # and against the definition, on the device
    assert wsi.norm2_noalloc(y) == pytest.approx(float(torch.linalg.vector_norm(y)), rel=1e-13)
    ctx.close()


def test_empty_and_oversized_inputs():
    L = wsi.lib()
    L.wsi_norm2_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_void_p]
    y = torch.ones(8, dtype=torch.float64, device="cuda")
    out = ctypes.c_double(-1.0)
    assert L.wsi_norm2_noalloc(ctypes.c_void_p(y.data_ptr()), 0, ctypes.byref(out), None) == wsi.OK
    assert out.value == 0.0
    # more elements than the static partial sums cover: rejected before any access
    rc = L.wsi_norm2_noalloc(ctypes.c_void_p(y.data_ptr()), 2 ** 27 + 1, ctypes.byref(out), None)
    assert rc == wsi.ERR_INVALID_ARG
    assert wsi.norm2_noalloc(y) == pytest.approx(np.sqrt(8.0), rel=1e-15)
    # host memory is refused before any launch, through the C ABI and the wrapper
    h = np.ones(8)
    rc = L.wsi_norm2_noalloc(ctypes.c_void_p(h.ctypes.data), 8, ctypes.byref(out), None)
    assert rc == wsi.ERR_INVALID_ARG
    with pytest.raises(TypeError):
        wsi.norm2_noalloc(h)
    # the context is still usable afterwards
    assert wsi.norm2_noalloc(y) == pytest.approx(np.sqrt(8.0), rel=1e-15)
