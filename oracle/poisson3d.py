"""ctypes wrapper of the 3D pressure-Poisson oracle (poisson3d.c) -- TEST
INFRASTRUCTURE ONLY.

Arrays are numpy FP64 with x fastest: cells (nz, ny, nx); beta_x (nz, ny, nx+1);
beta_y (nz, ny+1, nx); beta_z (nz+1, ny, nx).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import tank as _tank

_dp = C.POINTER(C.c_double)
_done = False


def _lib():
    global _done
    L = _tank.lib()
    if not _done:
        L.oracle3_poisson_apply.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.oracle3_poisson_apply.restype = None
        L.oracle3_levels.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.oracle3_vcycle.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.c_int, C.c_int, _dp, _dp]
        L.oracle3_poisson_solve.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double,
                                            C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_double)]
        _done = True
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _check(bx, by, bz, shape):
    nz, ny, nx = shape
    assert bx.shape == (nz, ny, nx + 1) and by.shape == (nz, ny + 1, nx) and bz.shape == (nz + 1, ny, nx)
    return nx, ny, nz


def apply(bx, by, bz, x):
    """y = A x."""
    bx, by, bz, x = _f64(bx), _f64(by), _f64(bz), _f64(x)
    nx, ny, nz = _check(bx, by, bz, x.shape)
    y = np.zeros_like(x)
    _lib().oracle3_poisson_apply(nx, ny, nz, _ptr(bx), _ptr(by), _ptr(bz), _ptr(x), _ptr(y))
    return y


def levels(nx, ny, nz):
    """(number of multigrid levels, coarsest (nx, ny, nz))."""
    out = (C.c_int * 3)()
    nl = _lib().oracle3_levels(nx, ny, nz, out)
    return nl, tuple(out)


def vcycle(bx, by, bz, b, nu1=2, nu2=2):
    """x = M^{-1} b (one V-cycle from zero); returns (x, levels)."""
    bx, by, bz, b = _f64(bx), _f64(by), _f64(bz), _f64(b)
    nx, ny, nz = _check(bx, by, bz, b.shape)
    x = np.zeros_like(b)
    nl = _lib().oracle3_vcycle(nx, ny, nz, _ptr(bx), _ptr(by), _ptr(bz), nu1, nu2, _ptr(b), _ptr(x))
    return x, nl


def solve(bx, by, bz, b, x0=None, rtol=1e-10, maxit=500, restart=20, nu1=2, nu2=2):
    """FGMRES + V-cycle; returns (x, {iters, relres, status})."""
    bx, by, bz, b = _f64(bx), _f64(by), _f64(bz), _f64(b)
    nx, ny, nz = _check(bx, by, bz, b.shape)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it, rr = C.c_int(0), C.c_double(0.0)
    st = _lib().oracle3_poisson_solve(nx, ny, nz, _ptr(bx), _ptr(by), _ptr(bz), _ptr(b), _ptr(x), rtol, maxit,
                                      restart, nu1, nu2, C.byref(it), C.byref(rr))
    return x, dict(iters=it.value, relres=rr.value, status=st)
