"""Rigid-body projection of the DLM method (Sec. 4.2.5) and the structure
level set rebuilt from the markers (Sec. 4.1, centre-of-mass equation).

Oracle (test infrastructure only).

  X_com = mean of the body's marker positions
  R_l   = X_l - X_com
  free DOFs: M U_r = sum rho_s (J u~)_l dV,   I W_r = sum rho_s R_l x (J u~)_l dV,
             I = sum rho_s dV (R.R Id - R (x) R).  rho_s and dV are uniform in a
             body, so they cancel: U_r is the mean marker velocity and
             W_r solves (sum R.R Id - R(x)R) W = sum R x U.
             (Reading: the paper's printed inertia tensor omits dV; it is
             included here, and cancels the same way.)
  locked DOFs: the prescribed values replace the computed ones, per DOF.
  U_b = U_r + W_r x R_l
  u = u~ + S[X](U_b - J[X] u~)                 (velocity correction equation)
  X^{n+1,k+1} = X^n + dt (U_b^{n+1,k+1} + U_b^n)/2   (position update)
"""
import numpy as np

from .grid import Grid
from .ib import interpolate, spread


def rigid_fit(X, U):
    """Free-body U_r and W_r from marker positions X and velocities U."""
    Xc = X.mean(axis=0)
    R = X - Xc
    Ur = U.mean(axis=0)
    L = np.cross(R, U).sum(axis=0)
    rr = (R * R).sum(axis=1)
    I = np.eye(3) * rr.sum() - R.T @ R
    # a planar body (2-D run) has no inertia about in-plane axes only if all
    # markers are collinear; lstsq returns the minimum-norm solution then
    W = np.linalg.lstsq(I, L, rcond=None)[0]
    return Ur, W, Xc


def body_velocity(X, Xc, Ur, Wr):
    R = X - Xc
    return Ur[None, :] + np.cross(Wr[None, :], R)


def constrain(g: Grid, vel, X, dV, lock, U_pres, W_pres, full=False):
    """One rigidity projection for a single body.

    vel: (u, v, w) uncorrected velocity; X: marker positions used for J and S
    (X^{n+1/2,k}); lock: 6 booleans (Ux,Uy,Uz,Wx,Wy,Wz), True = prescribed.
    Returns corrected (u, v, w), U_b per marker, U_r, W_r, X_com (and, with
    full, the interpolated velocity J u~ per marker)."""
    Ui = interpolate(g, vel, X)
    Ur, Wr, Xc = rigid_fit(X, Ui)
    lock = np.asarray(lock, dtype=bool)
    Ur = np.where(lock[:3], U_pres, Ur)
    Wr = np.where(lock[3:], W_pres, Wr)
    Ub = body_velocity(X, Xc, Ur, Wr)
    corr = spread(g, Ub - Ui, X, dV)
    new = [vel[c] + corr[c] for c in range(3)]
    if full:
        return new, Ub, Ur, Wr, Xc, Ui
    return new, Ub, Ur, Wr, Xc


def lm_force(Ub_new, Ub_old, dU, rho_s, dV, dt):
    """Net hydrodynamic force on the body by the Lagrange-multiplier method
    (Sec. 8, the LM-force equation), summed over the markers:
        F^{n+1} = sum_l rho_s [(U_b^{n+1} - U_b^n)/dt - dU^{n+1}/dt] dV,
    dU = U_b - J u~ the rigidity correction of the last cycle."""
    return rho_s * dV * np.sum((Ub_new - Ub_old) / dt - dU / dt, axis=0)


def update_positions(Xn, Ub_new, Ub_old, dt):
    return Xn + dt * 0.5 * (Ub_new + Ub_old)
