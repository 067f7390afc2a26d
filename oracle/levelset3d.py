"""ctypes wrapper of the 3D level-set oracle (levelset3d.c) -- TEST
INFRASTRUCTURE ONLY.  ``cfg`` is a 3D workload dict (synth.tank3d); arrays are
numpy FP64, cells (nz, ny, nx), u (nz, ny, nx+1), v (nz, ny+1, nx), w (nz+1, ny, nx)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import tank as _tank
from . import waves as _waves

_dp = C.POINTER(C.c_double)


class Tank3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double), ("depth", C.c_double),
                ("rho_w", C.c_double), ("rho_a", C.c_double), ("mu_w", C.c_double), ("mu_a", C.c_double),
                ("ncomp", C.c_int), ("amp", _dp), ("omega", _dp), ("kwave", _dp), ("phase", _dp),
                ("damp_x0", C.c_double), ("damp_len", C.c_double),
                ("has_body", C.c_int), ("body_xc", C.c_double), ("body_yc", C.c_double), ("body_r", C.c_double),
                ("body_len", C.c_double), ("body_mass", C.c_double)]


_done = False


def _lib():
    global _done
    L = _tank.lib()
    if not _done:
        L.oracle3_materials.argtypes = [C.POINTER(Tank3), _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.oracle3_materials.restype = None
        L.oracle3_advect.argtypes = [C.POINTER(Tank3), _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.oracle3_advect.restype = None
        L.oracle3_reinit.argtypes = [C.POINTER(Tank3), _dp, C.c_int, C.c_double]
        L.oracle3_reinit.restype = None
        L.oracle3_advect_cells.argtypes = [C.POINTER(Tank3), _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                           C.POINTER(C.c_longlong), C.c_int, _dp]
        L.oracle3_advect_cells.restype = None
        L.oracle3_advect_half.argtypes = [C.POINTER(Tank3), _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                          C.c_double, _dp]
        L.oracle3_advect_half.restype = None
        _done = True
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Oracle3:
    """The 3D tank's parameters as the oracle takes them."""

    def __init__(self, cfg):
        self.cfg = cfg
        amp, omega, k, phase = _waves.components(cfg["wave"], cfg["depth"], cfg["g"])
        self._w = [_f64(amp), _f64(omega), _f64(k), _f64(phase)]
        P = Tank3()
        P.nx, P.ny, P.nz = cfg["nx"], cfg["ny"], cfg["nz"]
        P.h, P.depth = cfg["lx"] / cfg["nx"], cfg["depth"]
        P.rho_w, P.rho_a, P.mu_w, P.mu_a = cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"]
        P.ncomp = len(amp)
        P.amp, P.omega, P.kwave, P.phase = (_ptr(a) for a in self._w)
        P.damp_x0, P.damp_len = cfg["damp_x0"], cfg["damp_len"]
        b = cfg.get("body")
        P.has_body = 1 if b else 0
        if b:
            P.body_xc, P.body_yc, P.body_r, P.body_len, P.body_mass = b["xc"], b["yc"], b["radius"], b["length"], \
                b["mass"]
        self.P = P
        self.shape = (P.nz, P.ny, P.nx)

    def materials(self, sigma, zc):
        s = _f64(sigma)
        assert s.shape == self.shape
        out = [np.zeros(self.shape) for _ in range(4)]
        _lib().oracle3_materials(C.byref(self.P), _ptr(s), zc, *(_ptr(a) for a in out))
        return dict(zip(("rho", "mu", "rho_flow", "chi"), out))

    def advect(self, sigma, u, v, w, dt, t):
        s, u, v, w = _f64(sigma), _f64(u), _f64(v), _f64(w)
        nz, ny, nx = self.shape
        assert u.shape == (nz, ny, nx + 1) and v.shape == (nz, ny + 1, nx) and w.shape == (nz + 1, ny, nx)
        out = np.zeros(self.shape)
        _lib().oracle3_advect(C.byref(self.P), _ptr(s), _ptr(u), _ptr(v), _ptr(w), dt, t, _ptr(out))
        return out

    def advect_half(self, base, sigma, u, v, w, dt, ta, tb):
        """A fixed-point cycle's update: base - dt Q(u, sigma), then the damping
        blend; the inflow ghosts of sigma and w use the mean of times ta, tb."""
        b, s, u, v, w = _f64(base), _f64(sigma), _f64(u), _f64(v), _f64(w)
        nz, ny, nx = self.shape
        assert b.shape == s.shape == self.shape
        assert u.shape == (nz, ny, nx + 1) and v.shape == (nz, ny + 1, nx) and w.shape == (nz + 1, ny, nx)
        out = np.zeros(self.shape)
        _lib().oracle3_advect_half(C.byref(self.P), _ptr(b), _ptr(s), _ptr(u), _ptr(v), _ptr(w), dt, ta, tb,
                                   _ptr(out))
        return out

    def advect_cells(self, sigma, u, v, w, dt, t, cells):
        """The advected sigma at the listed flat cell indices only."""
        s, u, v, w = _f64(sigma), _f64(u), _f64(v), _f64(w)
        cl = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(len(cl))
        _lib().oracle3_advect_cells(C.byref(self.P), _ptr(s), _ptr(u), _ptr(v), _ptr(w), dt, t,
                                    cl.ctypes.data_as(C.POINTER(C.c_longlong)), len(cl), _ptr(out))
        return out

    def reinit(self, sigma, nit, t):
        s = _f64(sigma).copy()
        assert s.shape == self.shape
        _lib().oracle3_reinit(C.byref(self.P), _ptr(s), nit, t)
        return s
