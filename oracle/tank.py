"""ctypes wrapper of the C oracle -- TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build
from . import waves as _waves

_lib = None

F_SIGMA, F_U, F_V, F_P, F_USTAR, F_VSTAR, F_BETA_U, F_BETA_V, F_RHS, F_SIGMA_ADV, F_RHOB_U, F_RHOB_V = range(12)

_dp = C.POINTER(C.c_double)


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("depth", C.c_double),
        ("rho_w", C.c_double), ("rho_a", C.c_double), ("mu_w", C.c_double), ("mu_a", C.c_double),
        ("g", C.c_double),
        ("ncomp", C.c_int),
        ("amp", _dp), ("omega", _dp), ("kwave", _dp), ("phase", _dp),
        ("damp_x0", C.c_double), ("damp_len", C.c_double), ("probe_x", C.c_double),
        ("has_body", C.c_int),
        ("body_xc", C.c_double), ("body_yc", C.c_double), ("body_w", C.c_double), ("body_h", C.c_double),
        ("body_mass", C.c_double), ("added_mass", C.c_double), ("kappa_p", C.c_double), ("pto_damping", C.c_double),
        ("rtol", C.c_double),
        ("max_iters", C.c_int), ("restart", C.c_int), ("n_reinit", C.c_int), ("n_jacobi", C.c_int),
        ("mg_pre", C.c_int), ("mg_post", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("t", "z", "zdot", "f_hydro", "f_pto", "eta_probe", "residual", "div_norm")] + \
               [("iters", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NlfkParams(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("h", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("depth", C.c_double), ("rho_w", C.c_double), ("g", C.c_double), ("ncomp", C.c_int),
                ("amp", _dp), ("omega", _dp), ("kwave", _dp), ("phase", _dp),
                ("body_xc", C.c_double), ("body_w", C.c_double), ("body_h", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.oracle_threads.restype = C.c_int
        L.oracle_threads.argtypes = [C.c_int]
        L.oracle_create.restype = C.c_void_p
        L.oracle_create.argtypes = [C.POINTER(Params)]
        L.oracle_destroy.argtypes = [C.c_void_p]
        L.oracle_step.argtypes = [C.c_void_p, C.c_double, C.c_double, C.POINTER(Result)]
        L.oracle_get.argtypes = [C.c_void_p, C.c_int, _dp]
        L.oracle_set.argtypes = [C.c_void_p, C.c_int, _dp]
        L.oracle_get_body.argtypes = [C.c_void_p, _dp]
        L.oracle_set_body.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]
        L.oracle_advect.argtypes = [C.c_void_p, C.c_double]
        L.oracle_reinit.argtypes = [C.c_void_p, C.c_int]
        L.oracle_materials.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_heaviside.restype = C.c_double
        L.oracle_heaviside.argtypes = [C.c_double, C.c_double]
        L.oracle_inflow.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _dp]
        L.oracle_transport.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.oracle_viscous.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.oracle_force.restype = C.c_double
        L.oracle_force.argtypes = [C.c_void_p]
        L.oracle_poisson_apply.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        L.oracle_poisson_solve.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_int,
                                           C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                           C.POINTER(C.c_double)]
        L.oracle_vcycle.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, _dp, _dp]
        L.oracle_nlfk.argtypes = [C.POINTER(NlfkParams), C.c_double, C.c_double, C.c_int, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleTank:
    """One 2D tank stepped by the oracle.  ``cfg`` is a workload dict from synth."""

    def __init__(self, cfg):
        L = lib()
        self.cfg = cfg
        nx, ny = cfg["nx"], cfg["ny"]
        self.nx, self.ny = nx, ny
        amp, omega, k, phase = _waves.components(cfg["wave"], cfg["depth"], cfg["g"])
        self._waves = [_f64(amp), _f64(omega), _f64(k), _f64(phase)]
        s = cfg["solver"]
        b = cfg.get("body")
        P = Params()
        P.nx, P.ny, P.lx, P.ly, P.depth = nx, ny, cfg["lx"], cfg["ly"], cfg["depth"]
        P.rho_w, P.rho_a, P.mu_w, P.mu_a, P.g = cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"], cfg["g"]
        P.ncomp = len(amp)
        P.amp, P.omega, P.kwave, P.phase = (_ptr(a) for a in self._waves)
        P.damp_x0, P.damp_len, P.probe_x = cfg["damp_x0"], cfg["damp_len"], cfg["probe_x"]
        P.has_body = 1 if b else 0
        if b:
            P.body_xc, P.body_yc, P.body_w, P.body_h = b["xc"], b["yc"], b["width"], b["height"]
            P.body_mass, P.kappa_p, P.pto_damping = b["mass"], b["kappa_p"], b["pto_damping"]
            P.added_mass = b["added_mass"]
        else:
            P.body_w = P.body_h = P.body_mass = 1.0
            P.kappa_p = 1e-8
        P.rtol = s["rtol"]
        P.max_iters, P.restart, P.n_reinit, P.n_jacobi = s["max_iters"], s["restart"], s["n_reinit"], s["n_jacobi"]
        P.mg_pre, P.mg_post = s["mg_pre"], s["mg_post"]
        self._P = P
        self.h = L.oracle_create(C.byref(P))
        if not self.h:
            raise ValueError("oracle_create rejected the parameters")

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    def shape(self, f):
        nx, ny = self.nx, self.ny
        if f in (F_U, F_USTAR, F_BETA_U, F_RHOB_U):
            return (ny, nx + 1)
        if f in (F_V, F_VSTAR, F_BETA_V, F_RHOB_V):
            return (ny + 1, nx)
        return (ny, nx)

    def get(self, f):
        a = np.zeros(self.shape(f))
        lib().oracle_get(self.h, f, _ptr(a))
        return a

    def set(self, f, a):
        a = _f64(a)
        assert a.shape == self.shape(f)
        lib().oracle_set(self.h, f, _ptr(a))

    def body(self):
        a = np.zeros(5)
        lib().oracle_get_body(self.h, _ptr(a))
        return dict(t=a[0], yc=a[1], zdot=a[2], yc0=a[3], zdot_prev=a[4])

    def set_body(self, t, yc, zdot, zdot_prev=None):
        lib().oracle_set_body(self.h, t, yc, zdot, zdot if zdot_prev is None else zdot_prev)

    def step(self, dt, f_pto=0.0):
        r = Result()
        st = lib().oracle_step(self.h, dt, f_pto, C.byref(r))
        d = r.as_dict()
        d["status"] = st
        return d

    def advect(self, dt):
        lib().oracle_advect(self.h, dt)

    def reinit(self, n):
        lib().oracle_reinit(self.h, n)

    def materials(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().oracle_materials(self.h, *(_ptr(a) for a in out))
        return dict(zip(("rho", "mu", "rho_flow", "chi"), out))

    def inflow(self, x, y, t):
        a = np.zeros(2)
        lib().oracle_inflow(self.h, x, y, t, _ptr(a))
        return a[0], a[1]

    def transport(self, rho_cell, dt):
        rbu = np.zeros((self.ny, self.nx + 1)); cu = np.zeros_like(rbu)
        rbv = np.zeros((self.ny + 1, self.nx)); cv = np.zeros_like(rbv)
        lib().oracle_transport(self.h, _ptr(_f64(rho_cell)), dt, _ptr(rbu), _ptr(rbv), _ptr(cu), _ptr(cv))
        return rbu, rbv, cu, cv

    def viscous(self, mu_cell):
        lx = np.zeros((self.ny, self.nx + 1)); ly = np.zeros((self.ny + 1, self.nx))
        lib().oracle_viscous(self.h, _ptr(_f64(mu_cell)), _ptr(lx), _ptr(ly))
        return lx, ly

    def force(self):
        return lib().oracle_force(self.h)


def heaviside(phi, eps):
    return lib().oracle_heaviside(phi, eps)


def poisson_apply(bu, bv, x):
    ny, nx = x.shape
    bu, bv, x = _f64(bu), _f64(bv), _f64(x)
    y = np.zeros_like(x)
    lib().oracle_poisson_apply(nx, ny, _ptr(bu), _ptr(bv), _ptr(x), _ptr(y))
    return y


def poisson_solve(bu, bv, b, x0=None, rtol=1e-10, maxit=500, restart=20, nu1=2, nu2=2):
    ny, nx = b.shape
    bu, bv, b = _f64(bu), _f64(bv), _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib().oracle_poisson_solve(nx, ny, _ptr(bu), _ptr(bv), _ptr(b), _ptr(x), rtol, maxit, restart,
                                    nu1, nu2, C.byref(it), C.byref(rr))
    return x, dict(iters=it.value, relres=rr.value, status=st)


def vcycle(bu, bv, b, nu1=2, nu2=2):
    ny, nx = b.shape
    bu, bv, b = _f64(bu), _f64(bv), _f64(b)
    x = np.zeros_like(b)
    nl = lib().oracle_vcycle(nx, ny, _ptr(bu), _ptr(bv), nu1, nu2, _ptr(b), _ptr(x))
    return x, nl


def nlfk(region, depth, rho_w, g, amp, omega, kwave, phase, body, t, yc, mode):
    """Static-grid NLFK force (fx, fy) per unit span (oracle_nlfk).
    region = (x0, y0, h, nx, ny); body = (xc, width, height); mode 0: incident
    wave pressure, 1: hydrostatic (nonlinear buoyancy)."""
    arrs = [_f64(np.atleast_1d(np.asarray(a, dtype=np.float64))) for a in (amp, omega, kwave, phase)]
    x0, y0, h, nx, ny = region
    P = NlfkParams(x0, y0, h, nx, ny, depth, rho_w, g, len(arrs[0]), *[_ptr(a) for a in arrs], *body)
    fx, fy = C.c_double(0), C.c_double(0)
    lib().oracle_nlfk(C.byref(P), t, yc, mode, C.byref(fx), C.byref(fy))
    return fx.value, fy.value
