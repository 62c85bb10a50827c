"""Exact solution of the implicit Stokes system (Sec. 4.2.4).

Oracle (test infrastructure only).

The paper solves the conservative momentum and continuity equations
simultaneously with FGMRES preconditioned by a projection method; whatever
the solver, the result is the solution of the saddle system

        A u + G p = b_u,     -D u = b_p,

unique up to a constant in p in a closed box.  The oracle computes that
solution directly: it assembles K (by probing the matrix-free operator with
a 3-colouring of every component's index lattice; the stencil reaches one
index in each direction, so a colour class never has two columns feeding the
same row) and solves the system bordered with the constraint sum(p) = 0 by
sparse LU (scipy.sparse.linalg.spsolve, a library primitive).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid
from .operators import stokes_apply


def _index_tables(g: Grid):
    """Per packed entry: component, i, j, k."""
    comps, I, J, K = [], [], [], []
    shapes = [g.face_shape(0), g.face_shape(1), g.face_shape(2), g.cell_shape]
    for q, s in enumerate(shapes):
        kk, jj, ii = np.meshgrid(np.arange(s[0]), np.arange(s[1]), np.arange(s[2]), indexing="ij")
        comps.append(np.full(ii.size, q))
        I.append(ii.ravel())
        J.append(jj.ravel())
        K.append(kk.ravel())
    return shapes, np.concatenate(comps), np.concatenate(I), np.concatenate(J), np.concatenate(K)


def assemble(g: Grid, apply_fn, reach=1):
    """Sparse matrix of a local linear operator on packed Stokes vectors."""
    M = 2 * reach + 1
    shapes, comp, I, J, K = _index_tables(g)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in shapes])
    n = offs[-1]
    unk = g.unknown_mask()
    probes = []
    for q in range(4):
        sel = comp == q
        for a in range(M):
            for b in range(M):
                for c in range(M):
                    m = sel & unk & (I % M == a) & (J % M == b) & (K % M == c)
                    if m.any():
                        probes.append((q, a, b, c, m))
    X = np.zeros((len(probes), n))
    for t, (_, _, _, _, m) in enumerate(probes):
        X[t, m] = 1.0
    Y = apply_fn(X)
    rows, cols, vals = [], [], []
    for t, (q, a, b, c, _) in enumerate(probes):
        r = np.nonzero(Y[t])[0]
        if r.size == 0:
            continue
        di = (a - I[r] + reach) % M - reach
        dj = (b - J[r] + reach) % M - reach
        dk = (c - K[r] + reach) % M - reach
        ci, cj, ck = I[r] + di, J[r] + dj, K[r] + dk
        s = shapes[q]
        ok = (ci >= 0) & (ci < s[2]) & (cj >= 0) & (cj < s[1]) & (ck >= 0) & (ck < s[0])
        assert ok.all(), "operator reaches further than the colouring allows"
        col = offs[q] + (ck * s[1] + cj) * s[2] + ci
        assert unk[col].all()
        rows.append(r)
        cols.append(col)
        vals.append(Y[t, r])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A


def stokes_matrix(g: Grid, mat, rho_face, dt, theta):
    return assemble(g, lambda X: stokes_apply(g, mat, rho_face, dt, theta, X))


def solve_stokes(g: Grid, mat, rho_face, dt, theta, b):
    """Solution x = (u, v, w, p) of K x = b with sum(p) = 0, zero on wall faces.

    b is a packed Stokes vector (b_u on faces, b_p at cells); its wall-face
    entries are ignored.  Returns x packed.  With an open top the pressure
    is fixed by p = 0 on the top plane: no constraint on sum(p)."""
    Kfull = stokes_matrix(g, mat, rho_face, dt, theta)
    unk = np.nonzero(g.unknown_mask())[0]
    Ku = Kfull[unk][:, unk]
    nu = unk.size
    x = np.zeros(b.shape[-1])
    if g.open_top:
        x[unk] = spla.spsolve(sp.csc_matrix(Ku), b[unk])
        return x
    np_ = g.n_cells
    e = np.zeros(nu)
    e[nu - np_:] = 1.0  # pressure entries are last in the packing
    Kb = sp.bmat([[Ku, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    rhs = np.concatenate([b[unk], [0.0]])
    sol = spla.spsolve(Kb, rhs)
    x[unk] = sol[:nu]
    return x


def solve_stokes_inlet(g: Grid, mat, rho_face, dt, theta, b, u_in, w_in):
    """Solution of the Stokes system with a Dirichlet inlet on the x- side
    (Sec. 7.1): normal velocity u_in (nz, ny) on the x- faces, tangential
    velocity w_in (nz+1, ny) on the x- edges.  The data are lifted to the
    right-hand side: K x~ = b - K_in x_b with x_b zero except u_in on the x-
    faces and K_in the operator with the inlet's affine ghost; x = x~ + x_b."""
    u0 = np.zeros(g.face_shape(0))
    u0[..., 0] = u_in
    xb = g.pack(u0, np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2)), np.zeros(g.cell_shape))
    r = b - stokes_apply(g, mat, rho_face, dt, theta, xb, inlet_w=w_in)
    return solve_stokes(g, mat, rho_face, dt, theta, r) + xb
