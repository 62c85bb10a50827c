"""ctypes binding of libwsi (C ABI in include/wsi.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Array arguments may be numpy float64 arrays (host) or torch
float64 CUDA tensors (device); outputs are returned in the kind of the
first array argument.  Loading fails loudly when the library is missing:
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libwsi.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NAN, ERR_OOM, ERR_DEVICE = range(7)
PREC_FP64, PREC_MIXED = 0, 1
GRAVITY_FLOW, GRAVITY_FULL = 0, 1
F_VEL, F_P, F_PHI, F_PSI, F_MARKERS, F_VEL_OLD = range(6)
C_RHO_CC, C_MU_CC, C_RHO_FACE, C_RHO_FLOW_FACE, C_MU_EDGE = range(5)
OP_STOKES, OP_VISCOUS, OP_STRAIN, OP_PRESSURE, OP_GRAD, OP_DIV = range(6)

EXPORTED = ["wsi_stokes_size", "wsi_velocity_size", "wsi_create_grid", "wsi_destroy", "wsi_last_error",
            "wsi_set_phases", "wsi_stokes_solve", "wsi_dlm_constrain", "wsi_step", "wsi_get_field",
            "wsi_set_field", "wsi_get_coeff", "wsi_apply", "wsi_transport", "wsi_advect_levelset",
            "wsi_interp", "wsi_spread", "wsi_set_waves", "wsi_wave_relax", "wsi_launch_count",
            "wsi_ktimer_enable", "wsi_ktimer_read", "wsi_unet_create", "wsi_unet_destroy", "wsi_unet_num_params",
            "wsi_unet_set_params", "wsi_unet_get_params", "wsi_unet_get_grads", "wsi_unet_forward",
            "wsi_unet_backward", "wsi_unet_adam", "wsi_attach_unet", "wsi_unet_train_sample",
            "wsi_pressure_solve", "wsi_checkpoint", "wsi_restore", "wsi_unet_save", "wsi_unet_load",
            "wsi_norm2_noalloc", "wsi_reinit", "wsi_fma_peak", "wsi_ktimer_bytes", "wsi_attach_unet_guess",
            "wsi_unet_train_guess"]
FORM_CONSISTENT, FORM_NONCONSERVATIVE = 0, 1
SMOOTH_RBGS, SMOOTH_CHEBYSHEV = 0, 1
LIMIT_CUI, LIMIT_XSPPM7 = 0, 1
KC_STOKES, KC_RBGS_P, KC_RBGS_V, KC_TRANSPORT, KC_MDOT, KC_MAXPY, KC_RESTRICT, KC_PROLONG, KC_REINIT = range(9)


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc", ctypes.c_double * 6), ("gravity", ctypes.c_double * 3),
                ("n_cells", ctypes.c_double), ("theta", ctypes.c_double),
                ("precision", ctypes.c_int), ("mg_pre", ctypes.c_int), ("mg_post", ctypes.c_int),
                ("mg_cycles", ctypes.c_int), ("visc_sweeps", ctypes.c_int), ("restart", ctypes.c_int),
                ("visc_mg", ctypes.c_int), ("reinit_iters", ctypes.c_int), ("transport_form", ctypes.c_int),
                ("mg_smoother", ctypes.c_int), ("ls_limiter", ctypes.c_int), ("open_top", ctypes.c_int)]


class PhaseProps(ctypes.Structure):
    _fields_ = [("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double), ("rho_s", ctypes.c_double),
                ("mu_l", ctypes.c_double), ("mu_g", ctypes.c_double), ("mu_s", ctypes.c_double),
                ("gravity_mode", ctypes.c_int)]


class BodyDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n_markers", ctypes.c_int), ("dV", ctypes.c_double),
                ("lock", ctypes.c_int * 6), ("U_pres", ctypes.c_double * 3), ("W_pres", ctypes.c_double * 3),
                ("shape", ctypes.c_int), ("half", ctypes.c_double * 3)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iters", ctypes.c_int), ("use_x0", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms", ctypes.c_double),
                ("learned_rejected", ctypes.c_int), ("guess", ctypes.c_int)]


class BodyState(ctypes.Structure):
    _fields_ = [("U_r", ctypes.c_double * 3), ("W_r", ctypes.c_double * 3), ("X_com", ctypes.c_double * 3)]


class StepStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * 4), ("rel_residual", ctypes.c_double * 4),
                ("umax", ctypes.c_double), ("ms", ctypes.c_double), ("F_lm", ctypes.c_double * 3)]


class WaveDesc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("T", ctypes.c_double), ("depth", ctypes.c_double),
                ("x_gen", ctypes.c_double), ("x_damp", ctypes.c_double), ("t0", ctypes.c_double),
                ("vertical", ctypes.c_int), ("inlet", ctypes.c_int)]


class WsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libwsi error %d: %s" % (code, msg))
        self.code = code


def lib_path():
    return _LIB_PATH


def lib():
    """Load libwsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libwsi.so not built: run __graft_entry__.build() (no CPU fallback exists)")
    L = ctypes.CDLL(_LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.wsi_stokes_size.restype = ctypes.c_size_t
    L.wsi_stokes_size.argtypes = [vp]
    L.wsi_velocity_size.restype = ctypes.c_size_t
    L.wsi_velocity_size.argtypes = [vp]
    L.wsi_create_grid.argtypes = [ctypes.POINTER(GridDesc), vp, ctypes.POINTER(vp)]
    L.wsi_destroy.argtypes = [vp]
    L.wsi_destroy.restype = None
    L.wsi_last_error.argtypes = [vp]
    L.wsi_last_error.restype = ctypes.c_char_p
    L.wsi_set_phases.argtypes = [vp, vp, vp, ctypes.POINTER(PhaseProps), ctypes.POINTER(BodyDesc), ip]
    L.wsi_stokes_solve.argtypes = [vp, vp, vp, dp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats)]
    L.wsi_dlm_constrain.argtypes = [vp, vp, ctypes.POINTER(BodyState)]
    L.wsi_step.argtypes = [vp, dp, ctypes.POINTER(SolveOpts), ctypes.POINTER(StepStats)]
    L.wsi_get_field.argtypes = [vp, ip, vp]
    L.wsi_set_field.argtypes = [vp, ip, vp]
    L.wsi_get_coeff.argtypes = [vp, ip, vp]
    L.wsi_apply.argtypes = [vp, ip, vp, vp, dp]
    L.wsi_transport.argtypes = [vp, vp, vp, vp, ip, dp, vp, vp]
    L.wsi_advect_levelset.argtypes = [vp, vp, vp, vp, dp, vp]
    L.wsi_reinit.argtypes = [vp, vp, ip]
    L.wsi_interp.argtypes = [vp, vp, vp, ip, vp]
    L.wsi_spread.argtypes = [vp, vp, vp, ip, dp, vp]
    L.wsi_set_waves.argtypes = [vp, ctypes.POINTER(WaveDesc)]
    L.wsi_wave_relax.argtypes = [vp, dp, vp, vp]
    L.wsi_launch_count.argtypes = []
    L.wsi_launch_count.restype = ctypes.c_longlong
    L.wsi_ktimer_enable.argtypes = [ip]
    L.wsi_ktimer_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    for name in EXPORTED:
        if name not in ("wsi_destroy", "wsi_last_error", "wsi_stokes_size", "wsi_velocity_size",
                        "wsi_launch_count", "wsi_unet_destroy", "wsi_unet_num_params"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        assert a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], \
        "arrays must be C-contiguous float64"
    return ctypes.c_void_p(a.ctypes.data)


def _empty_like_kind(ref, n):
    if _is_torch(ref):
        import torch
        return torch.empty(n, dtype=torch.float64, device=ref.device)
    return np.empty(n, dtype=np.float64)


def _flat(a):
    if _is_torch(a):
        return a.reshape(-1).contiguous()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


class Context:
    """One grid, its coefficients, solver state and (optionally) one body."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, bc=(-1.0,) * 6, gravity=(0.0, 0.0, -9.81),
                 n_cells=2.0, theta=0.5, precision=PREC_FP64, mg_pre=2, mg_post=2, mg_cycles=1,
                 visc_sweeps=2, restart=20, stream=None, visc_mg=0, reinit_iters=0,
                 transport_form=FORM_CONSISTENT, mg_smoother=SMOOTH_RBGS, ls_limiter=LIMIT_CUI, open_top=0):
        L = lib()
        d = GridDesc(nx, ny, nz, lx, ly, lz, (ctypes.c_double * 6)(*bc), (ctypes.c_double * 3)(*gravity),
                     n_cells, theta, precision, mg_pre, mg_post, mg_cycles, visc_sweeps, restart, visc_mg,
                     reinit_iters, transport_form, mg_smoother, ls_limiter, int(open_top))
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else None
        rc = L.wsi_create_grid(ctypes.byref(d), st, ctypes.byref(h))
        if rc != OK:
            raise WsiError(rc, "wsi_create_grid failed")
        self._h = h
        self.L = L
        self.dims = (nx, ny, nz)
        self.nstk = L.wsi_stokes_size(h)
        self.nvel = L.wsi_velocity_size(h)
        self.ncell = nx * ny * nz
        self.n_markers = 0

    @classmethod
    def from_case(cls, case, **kw):
        kw.setdefault("open_top", int(getattr(case, "open_top", False)))
        return cls(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, case.bc, case.gravity,
                   case.n_cells, case.theta, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.L.wsi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise WsiError(rc, self.L.wsi_last_error(self._h).decode())
        return rc

    # ---------------------------------------------------------------- set-up
    def set_phases(self, phi, psi, rho_l, rho_g, rho_s, mu_l, mu_g, mu_s, gravity_mode=GRAVITY_FLOW,
                   markers=None, dV=0.0, lock=(1,) * 6, U_pres=(0, 0, 0), W_pres=(0, 0, 0), box_half=None,
                   cylinder=None):
        props = PhaseProps(rho_l, rho_g, rho_s, mu_l, mu_g, mu_s, gravity_mode)
        phi, psi = _flat(phi), _flat(psi)
        nb = 0
        body = BodyDesc()
        keep = None
        if markers is not None and len(markers) > 0:
            keep = _flat(markers)
            body.X = _ptr(keep).value
            body.n_markers = len(markers)
            body.dV = dV
            body.lock = (ctypes.c_int * 6)(*[int(b) for b in lock])
            body.U_pres = (ctypes.c_double * 3)(*U_pres)
            body.W_pres = (ctypes.c_double * 3)(*W_pres)
            if box_half is not None:
                body.shape = 1
                body.half = (ctypes.c_double * 3)(*box_half)
            elif cylinder is not None:
                body.shape = 2
                body.half = (ctypes.c_double * 3)(cylinder[0], cylinder[1], 0.0)
            nb = 1
            self.n_markers = len(markers)
        rc = self.L.wsi_set_phases(self._h, _ptr(phi), _ptr(psi), ctypes.byref(props), ctypes.byref(body), nb)
        self._check(rc)

    def set_case(self, case, rho_s=None, gravity_mode=None, with_body=True, **kw):
        gm = case.gravity_mode if gravity_mode is None else gravity_mode
        gmode = GRAVITY_FLOW if gm == "flow" else GRAVITY_FULL
        self.set_phases(case.phi, case.psi, case.rho_l, case.rho_g, case.rho_s if rho_s is None else rho_s,
                        case.mu_l, case.mu_g, case.mu_s, gmode,
                        markers=case.markers if with_body else None, dV=case.dV,
                        lock=[int(b) for b in case.lock],
                        box_half=case.box_half if with_body else None,
                        cylinder=case.extra.get("cylinder") if with_body else None, **kw)

    # ---------------------------------------------------------------- compute
    def solve(self, rhs, dt, rtol=1e-10, max_iters=200, x0=None):
        rhs = _flat(rhs)
        if x0 is not None:
            x = _flat(x0).copy() if not _is_torch(x0) else _flat(x0).clone()
        else:
            x = _empty_like_kind(rhs, self.nstk)
        o = SolveOpts(rtol, max_iters, 1 if x0 is not None else 0)
        s = SolveStats()
        rc = self.L.wsi_stokes_solve(self._h, _ptr(rhs), _ptr(x), dt, ctypes.byref(o), ctypes.byref(s))
        self._check(rc, allow=(ERR_NOT_CONVERGED,))
        return x, s

    def apply(self, op, arr, dt=1.0):
        arr = _flat(arr)
        nout = {OP_STOKES: self.nstk, OP_VISCOUS: self.nvel, OP_STRAIN: self.nvel, OP_PRESSURE: self.ncell,
                OP_GRAD: self.nvel, OP_DIV: self.ncell}[op]
        out = _empty_like_kind(arr, nout)
        self._check(self.L.wsi_apply(self._h, op, _ptr(arr), _ptr(out), dt))
        return out

    def coeff(self, which, like=None):
        nx, ny, nz = self.dims
        n = {C_RHO_CC: self.ncell, C_MU_CC: self.ncell, C_RHO_FACE: self.nvel, C_RHO_FLOW_FACE: self.nvel,
             C_MU_EDGE: (nx + 1) * (ny + 1) * nz + (nx + 1) * ny * (nz + 1) + nx * (ny + 1) * (nz + 1)}[which]
        out = np.empty(n) if like is None else _empty_like_kind(like, n)
        self._check(self.L.wsi_get_coeff(self._h, which, _ptr(out)))
        return out

    def dlm_constrain(self, vel):
        v = _flat(vel)
        v = v.copy() if not _is_torch(v) else v.clone()
        bs = BodyState()
        self._check(self.L.wsi_dlm_constrain(self._h, _ptr(v), ctypes.byref(bs)))
        return v, bs

    def step(self, dt, rtol=1e-8, max_iters=100):
        o = SolveOpts(rtol, max_iters, 1)
        s = StepStats()
        self._check(self.L.wsi_step(self._h, dt, ctypes.byref(o), ctypes.byref(s)))
        return s

    def get_field(self, which, like=None):
        n = {F_VEL: self.nvel, F_VEL_OLD: self.nvel, F_P: self.ncell, F_PHI: self.ncell, F_PSI: self.ncell,
             F_MARKERS: 3 * self.n_markers}[which]
        out = np.empty(n) if like is None else _empty_like_kind(like, n)
        self._check(self.L.wsi_get_field(self._h, which, _ptr(out)))
        return out

    def set_field(self, which, arr):
        a = _flat(arr)
        self._check(self.L.wsi_set_field(self._h, which, _ptr(a)))

    def transport(self, u_n, u_nm1, u_k, k, dt):
        u_n, u_nm1 = _flat(u_n), _flat(u_nm1)
        u_k = _flat(u_k) if u_k is not None else u_n
        rho = _empty_like_kind(u_n, self.nvel)
        C = _empty_like_kind(u_n, self.nvel)
        self._check(self.L.wsi_transport(self._h, _ptr(u_n), _ptr(u_nm1), _ptr(u_k), k, dt, _ptr(rho), _ptr(C)))
        return rho, C

    def advect_levelset(self, vel, phi_n, phi_half, dt):
        vel, phi_n, phi_half = _flat(vel), _flat(phi_n), _flat(phi_half)
        out = _empty_like_kind(phi_n, self.ncell)
        self._check(self.L.wsi_advect_levelset(self._h, _ptr(vel), _ptr(phi_n), _ptr(phi_half), dt, _ptr(out)))
        return out

    def reinit(self, phi, iters):
        """Level-set reinitialisation (Sec. 4.1); returns the new level set
        (a copy: the argument is left unchanged)."""
        out = _flat(phi)
        out = out.clone() if _is_torch(out) else out.copy()
        self._check(self.L.wsi_reinit(self._h, _ptr(out), int(iters)))
        return out

    def checkpoint(self, path):
        self.L.wsi_checkpoint.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
        self._check(self.L.wsi_checkpoint(self._h, str(path).encode()))

    def restore(self, path):
        self.L.wsi_restore.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
        self._check(self.L.wsi_restore(self._h, str(path).encode()))

    def set_waves(self, H, T, depth, x_gen, x_damp, t0=0.0, vertical=2, inlet=False):
        w = WaveDesc(H, T, depth, x_gen, x_damp, t0, vertical, int(inlet))
        self._check(self.L.wsi_set_waves(self._h, ctypes.byref(w)))

    def wave_relax(self, t, vel, phi):
        v = _flat(vel)
        v = v.copy() if not _is_torch(v) else v.clone()
        p = _flat(phi)
        p = p.copy() if not _is_torch(p) else p.clone()
        self._check(self.L.wsi_wave_relax(self._h, t, _ptr(v), _ptr(p)))
        return v, p

    def interp(self, vel, X):
        vel, X = _flat(vel), _flat(X)
        n = X.shape[0] // 3
        U = _empty_like_kind(vel, 3 * n)
        self._check(self.L.wsi_interp(self._h, _ptr(vel), _ptr(X), n, _ptr(U)))
        return U

    def spread(self, F, X, dV):
        F, X = _flat(F), _flat(X)
        n = X.shape[0] // 3
        out = _empty_like_kind(F, self.nvel)
        self._check(self.L.wsi_spread(self._h, _ptr(F), _ptr(X), n, dV, _ptr(out)))
        return out


def norm2_noalloc(x, stream=None):
    """Float64 2-norm of a contiguous float64 CUDA tensor through the
    allocation-free entry point (run with the tensor's device current)."""
    if not (_is_torch(x) and x.is_cuda and x.dtype.is_floating_point and x.element_size() == 8
            and x.is_contiguous()):
        raise TypeError("norm2_noalloc takes a contiguous float64 CUDA tensor")
    import torch
    L = lib()
    L.wsi_norm2_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_void_p]
    L.wsi_norm2_noalloc.restype = ctypes.c_int
    out = ctypes.c_double()
    with torch.cuda.device(x.device):
        rc = L.wsi_norm2_noalloc(_ptr(x), int(x.numel()), ctypes.byref(out), stream)
    if rc != OK:
        raise WsiError(rc, "wsi_norm2_noalloc failed")
    return out.value


def fma_peak(fp64=True, stream=None, packed=False):
    """Measured FMA rate of the current GPU, GFLOP/s (float64, float32, or
    float32 issued as packed pairs)."""
    L = lib()
    L.wsi_fma_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    g = ctypes.c_double()
    rc = L.wsi_fma_peak(2 if packed else (1 if fp64 else 0), stream, ctypes.byref(g))
    if rc != OK:
        raise WsiError(rc, "wsi_fma_peak")
    return g.value


def launch_count():
    return int(lib().wsi_launch_count())


def ktimer_enable(kernel_class):
    rc = lib().wsi_ktimer_enable(kernel_class)
    if rc != OK:
        raise WsiError(rc, "wsi_ktimer_enable")


def ktimer_bytes():
    L = lib()
    L.wsi_ktimer_bytes.argtypes = [ctypes.POINTER(ctypes.c_double)]
    b = ctypes.c_double()
    rc = L.wsi_ktimer_bytes(ctypes.byref(b))
    if rc != OK:
        raise WsiError(rc, "wsi_ktimer_bytes")
    return b.value


def ktimer_read():
    t = ctypes.c_double()
    n = ctypes.c_longlong()
    rc = lib().wsi_ktimer_read(ctypes.byref(t), ctypes.byref(n))
    if rc != OK:
        raise WsiError(rc, "wsi_ktimer_read")
    return t.value, n.value


# ------------------------------------------------------------------ learned correction
_UNET_SIGS = False


def _unet_sigs():
    global _UNET_SIGS
    if _UNET_SIGS:
        return
    L = lib()
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.wsi_unet_create.argtypes = [ip, ip, ip, ip, ip, ip, ctypes.c_ulonglong, ctypes.POINTER(vp)]
    L.wsi_unet_create.restype = ip
    L.wsi_unet_destroy.argtypes = [vp]
    L.wsi_unet_destroy.restype = None
    L.wsi_unet_num_params.argtypes = [vp]
    L.wsi_unet_num_params.restype = ctypes.c_size_t
    for name in ("wsi_unet_set_params", "wsi_unet_get_params", "wsi_unet_get_grads"):
        getattr(L, name).argtypes = [vp, vp]
        getattr(L, name).restype = ip
    L.wsi_unet_forward.argtypes = [vp, vp, vp]
    L.wsi_unet_forward.restype = ip
    L.wsi_unet_backward.argtypes = [vp, vp, ctypes.POINTER(dp)]
    L.wsi_unet_backward.restype = ip
    L.wsi_unet_adam.argtypes = [vp, dp]
    L.wsi_unet_adam.restype = ip
    L.wsi_attach_unet.argtypes = [vp, vp, ip, ip]
    L.wsi_attach_unet.restype = ip
    L.wsi_unet_train_sample.argtypes = [vp, vp, dp, ctypes.POINTER(dp)]
    L.wsi_unet_train_sample.restype = ip
    L.wsi_pressure_solve.argtypes = [vp, vp, vp, dp, ip, ctypes.POINTER(SolveStats)]
    L.wsi_pressure_solve.restype = ip
    L.wsi_attach_unet_guess.argtypes = [vp, vp, ip]
    L.wsi_attach_unet_guess.restype = ip
    L.wsi_unet_train_guess.argtypes = [vp, vp, vp, dp, ctypes.POINTER(dp)]
    L.wsi_unet_train_guess.restype = ip
    _UNET_SIGS = True


def _fptr(a):
    assert isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


class UNet:
    """The learned correction network (float32 host arrays in and out)."""

    def __init__(self, nz, ny, nx, c0=16, c1=32, c2=64, seed=0):
        _unet_sigs()
        self.L = lib()
        h = ctypes.c_void_p()
        rc = self.L.wsi_unet_create(nz, ny, nx, c0, c1, c2, seed, ctypes.byref(h))
        if rc != OK:
            raise WsiError(rc, "wsi_unet_create failed")
        self._h = h
        self.dims = (nz, ny, nx)
        self.n = int(self.L.wsi_unet_num_params(h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.L.wsi_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, what):
        if rc != OK:
            raise WsiError(rc, what)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n
        self._ck(self.L.wsi_unet_set_params(self._h, _fptr(p)), "set_params")

    def params(self):
        p = np.empty(self.n, np.float32)
        self._ck(self.L.wsi_unet_get_params(self._h, _fptr(p)), "get_params")
        return p

    def grads(self):
        g = np.empty(self.n, np.float32)
        self._ck(self.L.wsi_unet_get_grads(self._h, _fptr(g)), "get_grads")
        return g

    def forward(self, x):
        """x: float32 [Z][Y][X][3] -> out [Z][Y][X]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty(self.dims, np.float32)
        self._ck(self.L.wsi_unet_forward(self._h, _fptr(x), _fptr(out)), "forward")
        return out

    def backward(self, target):
        t = np.ascontiguousarray(target, dtype=np.float32)
        loss = ctypes.c_double()
        self._ck(self.L.wsi_unet_backward(self._h, _fptr(t), ctypes.byref(loss)), "backward")
        return loss.value

    def adam(self, lr):
        self._ck(self.L.wsi_unet_adam(self._h, lr), "adam")

    def save(self, path):
        self.L.wsi_unet_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
        self._ck(self.L.wsi_unet_save(self._h, str(path).encode()), "save")

    def load(self, path):
        self.L.wsi_unet_load.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
        self._ck(self.L.wsi_unet_load(self._h, str(path).encode()), "load")


LEARN_OFF, LEARN_REPLACE, LEARN_AUGMENT = 0, 1, 2


def attach_unet(ctx, net, level, enable=LEARN_REPLACE):
    """enable: LEARN_OFF, LEARN_REPLACE or LEARN_AUGMENT (True = replace)."""
    _unet_sigs()
    mode = int(enable) if not isinstance(enable, bool) else (LEARN_REPLACE if enable else LEARN_OFF)
    ctx._check(ctx.L.wsi_attach_unet(ctx._h, net._h if net is not None else None, level, mode))


def attach_unet_guess(ctx, net, level):
    """Initial-guess network for pressure_solve (None detaches)."""
    _unet_sigs()
    ctx._check(ctx.L.wsi_attach_unet_guess(ctx._h, net._h if net is not None else None, level))


def unet_train_guess(ctx, y, x, lr):
    """One Adam step of the guess network on a solver-generated pair (fine
    right-hand side y, its solution x)."""
    _unet_sigs()
    y, x = _flat(y), _flat(x)
    loss = ctypes.c_double()
    ctx._check(ctx.L.wsi_unet_train_guess(ctx._h, _ptr(y), _ptr(x), lr, ctypes.byref(loss)))
    return loss.value


def unet_train_sample(ctx, e, lr):
    _unet_sigs()
    e = np.ascontiguousarray(e, dtype=np.float64)
    loss = ctypes.c_double()
    ctx._check(ctx.L.wsi_unet_train_sample(ctx._h, _ptr(e), lr, ctypes.byref(loss)))
    return loss.value


def pressure_solve(ctx, y, rtol=1e-8, max_cycles=200):
    _unet_sigs()
    y = _flat(y)
    x = _empty_like_kind(y, ctx.ncell)
    s = SolveStats()
    rc = ctx.L.wsi_pressure_solve(ctx._h, _ptr(y), _ptr(x), rtol, max_cycles, ctypes.byref(s))
    ctx._check(rc, allow=(ERR_NOT_CONVERGED,))
    return x, s
