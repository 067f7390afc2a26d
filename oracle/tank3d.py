"""ctypes wrapper of the 3D tank-step oracle (tank3d.c) -- TEST INFRASTRUCTURE
ONLY.  ``cfg`` is a 3D workload dict (synth.tank3d); fields are numpy FP64
arrays, cells (nz, ny, nx), u (nz, ny, nx+1), v (nz, ny+1, nx), w (nz+1, ny, nx)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import levelset3d as _ls
from . import tank as _tank

_dp = C.POINTER(C.c_double)
F_SIGMA, F_U, F_V, F_W, F_P = range(5)


class Params3(C.Structure):
    _fields_ = [("L", _ls.Tank3), ("g", C.c_double), ("kappa_p", C.c_double), ("added_mass", C.c_double),
                ("pto_damping", C.c_double), ("probe_x", C.c_double), ("lz", C.c_double), ("rtol", C.c_double),
                ("max_iters", C.c_int), ("restart", C.c_int), ("n_reinit", C.c_int), ("n_jacobi", C.c_int),
                ("mg_pre", C.c_int), ("mg_post", C.c_int), ("n_cycles", C.c_int)]


class Result3(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("t", "z", "zdot", "f_hydro", "f_pto", "eta_probe", "residual",
                                          "div_norm", "rhs_norm")] + [("iters", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_done = False


def _lib():
    global _done
    L = _tank.lib()
    if not _done:
        L.oracle3_create.restype = C.c_void_p
        L.oracle3_create.argtypes = [C.POINTER(Params3), C.c_double]
        L.oracle3_destroy.argtypes = [C.c_void_p]
        L.oracle3_destroy.restype = None
        L.oracle3_step.argtypes = [C.c_void_p, C.c_double, C.c_double, C.POINTER(Result3)]
        L.oracle3_get.argtypes = [C.c_void_p, C.c_int, _dp]
        L.oracle3_set.argtypes = [C.c_void_p, C.c_int, _dp]
        L.oracle3_get_body.argtypes = [C.c_void_p, _dp]
        L.oracle3_get_body.restype = None
        L.oracle3_force.argtypes = [C.c_void_p]
        L.oracle3_force.restype = C.c_double
        _done = True
    return L


class OracleTank3:
    """One 3D tank stepped by the oracle."""

    def __init__(self, cfg):
        self.cfg = cfg
        self._o = _ls.Oracle3(cfg)  # holds the wave arrays the parameters point to
        P = Params3()
        P.L = self._o.P
        b = cfg.get("body")
        s = cfg["solver"]
        P.g, P.kappa_p = cfg["g"], (b["kappa_p"] if b else 1e-8)
        P.added_mass = b["added_mass"] if b else 0.0
        P.pto_damping = b.get("pto_damping", 0.0) if b else 0.0
        P.probe_x, P.lz, P.rtol = cfg["probe_x"], cfg["lz"], s["rtol"]
        P.max_iters, P.restart, P.n_reinit, P.n_jacobi = s["max_iters"], s["restart"], s["n_reinit"], s["n_jacobi"]
        P.mg_pre, P.mg_post = s["mg_pre"], s["mg_post"]
        P.n_cycles = s.get("n_cycles", 1)
        self._P = P
        nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
        self.shapes = {F_SIGMA: (nz, ny, nx), F_U: (nz, ny, nx + 1), F_V: (nz, ny + 1, nx), F_W: (nz + 1, ny, nx),
                       F_P: (nz, ny, nx)}
        self.h = _lib().oracle3_create(C.byref(P), b["zc"] if b else 0.0)
        if not self.h:
            raise ValueError("oracle3_create failed")

    def __del__(self):
        if getattr(self, "h", None):
            _lib().oracle3_destroy(self.h)
            self.h = None

    def get(self, f):
        a = np.zeros(self.shapes[f])
        _lib().oracle3_get(self.h, f, a.ctypes.data_as(_dp))
        return a

    def set(self, f, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == self.shapes[f]
        _lib().oracle3_set(self.h, f, a.ctypes.data_as(_dp))

    def body(self):
        a = np.zeros(5)
        _lib().oracle3_get_body(self.h, a.ctypes.data_as(_dp))
        return dict(t=a[0], zc=a[1], zdot=a[2], zc0=a[3], zdot_prev=a[4])

    def force(self):
        return _lib().oracle3_force(self.h)

    def step(self, dt, f_pto=0.0):
        r = Result3()
        st = _lib().oracle3_step(self.h, dt, f_pto, C.byref(r))
        d = r.as_dict()
        d["status"] = st
        return d
