"""Plain FP64 CPU oracle for the implicit Stokes step of the DLM level-set
wave-structure-interaction method (Nangia, Patankar & Bhalla, arXiv 1901.07892).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA library; both sides receive the same seeded inputs from
``paper_1901_07892_gb300/inputs.py``, which holds no arithmetic of the method.

Every function is a literal, slow restatement of the paper's formulas in numpy
(vectorised slices, no blocking, no fusion).  Library primitives used as steps:
``scipy.sparse.linalg.spsolve`` (direct solve of the assembled saddle system),
``numpy.linalg.solve`` (3x3 inertia systems).

Modules
-------
grid        staggered MAC grid, index conventions, boundary-condition signs
materials   smoothed Heaviside and two-stage material properties (Sec. 4.1, Sec. 5)
operators   grad, div, pressure and viscous operators, Stokes matvec (Sec. 3.1, 4.2.2)
solve       exact solution of the saddle system (Sec. 4.2.4: the result FGMRES reaches)
ib          IB4 kernel, interpolation J and spreading S with boundary folding (Sec. 3.3)
rigid       rigid-body projection and momentum redistribution (Sec. 4.2.5)
transport   SSP-RK3 face-density update and consistent convective operator (Sec. 4.2.2)
levelset    conservative limited level-set advection (Sec. 4.2.1, stand-in limiter)
waves       second-order Stokes wave and relaxation zones (Sec. 7.1)
step        one full time step (Sec. 4.2)
"""
