"""ctypes binding of libwec (include/wec.h): argument marshalling only.

Every step of the wave-tank path runs in the CUDA library; there is no CPU
fallback.  Loading fails loudly if libwec.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwec.so")

WEC_OK, WEC_ERR_INVALID, WEC_ERR_CUDA, WEC_ERR_NOT_CONVERGED, WEC_ERR_NONFINITE, WEC_ERR_NOMEM = range(6)
PREC_FP64, PREC_MIXED, PREC_MIXED_MG, PREC_MIXED_DF = 0, 1, 2, 3
(F_SIGMA, F_U, F_V, F_P, F_USTAR, F_VSTAR, F_BETA_U, F_BETA_V, F_RHS, F_SIGMA_ADV) = range(10)
FIELD_NAMES = {"sigma": F_SIGMA, "u": F_U, "v": F_V, "p": F_P, "ustar": F_USTAR, "vstar": F_VSTAR,
               "beta_u": F_BETA_U, "beta_v": F_BETA_V, "rhs": F_RHS, "sigma_adv": F_SIGMA_ADV}

_dp = C.POINTER(C.c_double)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double), ("depth", C.c_double)]


class Fluids(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("rho_w", "rho_a", "mu_w", "mu_a", "g")]


class Waves(C.Structure):
    _fields_ = [("ncomp", C.c_int), ("amp", _dp), ("omega", _dp), ("phase", _dp),
                ("damp_x0", C.c_double), ("damp_len", C.c_double), ("probe_x", C.c_double)]


class Grid3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lz", C.c_double), ("depth", C.c_double)]


class Cylinder(C.Structure):
    _fields_ = [("present", C.c_int)] + [(k, C.c_double) for k in ("xc", "yc", "radius", "length", "mass", "zc",
                                                                   "kappa_p", "added_mass", "pto_damping")]


F3_SIGMA, F3_U, F3_V, F3_W, F3_RHO, F3_MU, F3_RHO_FLOW, F3_CHI, F3_P = range(9)


class Region(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("h", C.c_double), ("nx", C.c_int), ("ny", C.c_int)]


class Body(C.Structure):
    _fields_ = [("present", C.c_int)] + [(k, C.c_double) for k in
                                         ("xc", "yc", "width", "height", "mass", "added_mass", "kappa_p",
                                          "pto_damping")]


class SolverOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("rtol", C.c_double), ("max_iters", C.c_int), ("restart", C.c_int),
                ("n_reinit", C.c_int), ("n_jacobi", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int),
                ("n_cycles", C.c_int)]


class StepResult(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("t", "z", "zdot", "f_hydro", "f_pto", "eta_probe", "residual", "div_norm")] + \
               [("iters", C.c_int), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class WecError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libwec error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libwec.so (built by paper_2206_07732_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2206_07732_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.wec_last_error.restype = C.c_char_p
    L.wec_tank_create.argtypes = [C.POINTER(Grid), C.POINTER(Fluids), C.POINTER(Waves), C.POINTER(Body),
                                  C.POINTER(SolverOpts), vp, C.POINTER(vp)]
    L.wec_tank_destroy.argtypes = [vp]
    L.wec_tank_destroy.restype = None
    L.wec_step.argtypes = [vp, C.c_double, C.c_double, C.POINTER(StepResult)]
    L.wec_step_n.argtypes = [vp, C.c_int, C.c_double, _dp, C.POINTER(StepResult)]
    L.wec_batch_create.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(Fluids), C.POINTER(Waves), C.POINTER(Body),
                                   C.POINTER(SolverOpts), vp, C.POINTER(vp)]
    L.wec_batch_size.argtypes = [vp]
    L.wec_batch_tank.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.wec_batch_step.argtypes = [vp, _dp, _dp, C.POINTER(StepResult)]
    L.wec_batch_step_n.argtypes = [vp, C.c_int, _dp, _dp, C.POINTER(StepResult)]
    L.wec_batch_destroy.argtypes = [vp]
    L.wec_batch_destroy.restype = None
    L.wec_nlfk_create.argtypes = [C.POINTER(Region), C.POINTER(Fluids), C.c_double, C.POINTER(Waves), C.POINTER(Body),
                                  vp, C.POINTER(vp)]
    L.wec_nlfk_force.argtypes = [vp, C.c_double, C.c_double, C.c_int, _dp, _dp]
    L.wec_nlfk_destroy.argtypes = [vp]
    L.wec_nlfk_destroy.restype = None
    L.wec_pressure_solve.argtypes = [vp, vp, vp, C.c_double, C.POINTER(C.c_int), _dp]
    L.wec_tank_use_graph.argtypes = [vp, C.c_int]
    L.wec_set_option.argtypes = [C.c_char_p, C.c_int]
    L.wec_tank_mg_tiles.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    L.wec_launch_count.restype = C.c_longlong
    L.wec_profile_enable.argtypes = [C.c_int, C.c_char_p]
    L.wec_profile_read.argtypes = [C.c_int, C.c_char_p, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.wec_get_field.argtypes = [vp, C.c_int, _dp, C.c_size_t]
    L.wec_set_field.argtypes = [vp, C.c_int, _dp, C.c_size_t]
    L.wec_get_state.argtypes = [vp, _dp]
    L.wec_set_state.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
    L.wec_save.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.wec_load.argtypes = [vp, vp, C.c_size_t]
    L.wec_poisson_create.argtypes = [C.c_int, C.c_int, C.POINTER(SolverOpts), vp, C.POINTER(vp)]
    L.wec_poisson_destroy.argtypes = [vp]
    L.wec_poisson_destroy.restype = None
    L.wec_poisson_set_coefficients.argtypes = [vp, vp, vp]
    L.wec_poisson_apply.argtypes = [vp, vp, vp]
    L.wec_poisson_vcycle.argtypes = [vp, vp, vp]
    L.wec_poisson_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(C.c_int), _dp]
    L.wec_poisson_create3.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(SolverOpts), vp, C.POINTER(vp)]
    L.wec_tank3_create.argtypes = [C.POINTER(Grid3), C.POINTER(Fluids), C.POINTER(Waves), C.POINTER(Cylinder),
                                   C.POINTER(SolverOpts), vp, C.POINTER(vp)]
    L.wec_tank3_step.argtypes = [vp, C.c_double, C.c_double, C.POINTER(StepResult)]
    L.wec_tank3_get_state.argtypes = [vp, _dp]
    L.wec_tank3_destroy.argtypes = [vp]
    L.wec_tank3_destroy.restype = None
    L.wec_tank3_get_field.argtypes = [vp, C.c_int, _dp, C.c_size_t]
    L.wec_tank3_set_field.argtypes = [vp, C.c_int, _dp, C.c_size_t]
    L.wec_tank3_materials.argtypes = [vp, C.c_double]
    L.wec_tank3_advect.argtypes = [vp, C.c_double, C.c_double]
    L.wec_tank3_reinit.argtypes = [vp, C.c_int, C.c_double]
    L.wec_poisson_set_coefficients3.argtypes = [vp, vp, vp, vp]
    L.wec_wave_number.restype = C.c_double
    L.wec_wave_number.argtypes = [C.c_double, C.c_double, C.c_double]
    L.wec_wave_number_fenton_kd.restype = C.c_double
    L.wec_wave_number_fenton_kd.argtypes = [C.c_double, C.c_double, C.c_double]
    L.wec_jonswap.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp]
    _fp = C.POINTER(C.c_float)
    L.wec_net_param_count.restype = C.c_size_t
    L.wec_net_create.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.POINTER(vp)]
    L.wec_net_destroy.argtypes = [vp]
    L.wec_net_destroy.restype = None
    L.wec_net_set_params.argtypes = [vp, _fp, C.c_size_t]
    L.wec_net_get_params.argtypes = [vp, _fp, C.c_size_t]
    L.wec_net_get_grads.argtypes = [vp, _fp, C.c_size_t]
    L.wec_net_get_activation.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_uint16), C.c_size_t]
    L.wec_net_forward.argtypes = [vp, C.c_int, vp, vp]
    L.wec_net_loss_grad.argtypes = [vp, C.c_int, vp, vp, _dp]
    L.wec_net_adam.argtypes = [vp, C.c_float]
    L.wec_net_train_step.argtypes = [vp, vp, vp, C.POINTER(C.c_int), C.c_int, C.c_float, _dp]
    L.wec_net_sample.argtypes = [vp, vp, vp]
    L.wec_check_conversions.argtypes = [C.c_longlong, vp, vp, vp]
    L.wec_tank_set_net.argtypes = [vp, vp]
    L.wec_tank_net_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    _lib = L
    return L


def _check(code, ok=(WEC_OK,)):
    if code not in ok:
        raise WecError(code, load().wec_last_error().decode())
    return code


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _dev(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _dev32(t):
    """Device pointer of a contiguous float32 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def wave_number(omega, depth, g):
    return load().wec_wave_number(omega, depth, g)


def wave_number_fenton_kd(omega, depth, g):
    return load().wec_wave_number_fenton_kd(omega, depth, g)


def jonswap(Hs, Tp, gamma, ncomp):
    amp = np.zeros(ncomp)
    om = np.zeros(ncomp)
    _check(load().wec_jonswap(Hs, Tp, gamma, ncomp, _ptr(amp), _ptr(om)))
    return amp, om


def wave_components(wave):
    """(amp, omega, phase) of a workload's wave dict (JONSWAP built by the library)."""
    if wave["kind"] == "regular":
        return (np.array([0.5 * wave["H"]]), np.array([2.0 * math.pi / wave["T"]]),
                np.array([wave["phase"]], dtype=np.float64))
    if wave["kind"] == "jonswap":
        amp, om = jonswap(wave["Hs"], wave["Tp"], wave["gamma"], wave["ncomp"])
        return amp, om, np.asarray(wave["phases"], dtype=np.float64)
    raise ValueError(wave["kind"])


def solver_opts(s, precision=None):
    o = SolverOpts()
    o.precision = s.get("precision", 0) if precision is None else precision
    o.rtol = s["rtol"]
    o.max_iters, o.restart = s["max_iters"], s["restart"]
    o.n_reinit, o.n_jacobi, o.mg_pre, o.mg_post = s["n_reinit"], s["n_jacobi"], s["mg_pre"], s["mg_post"]
    o.n_cycles = s.get("n_cycles", 1)
    return o


def tank_structs(cfg, precision=None):
    """(grid, fluids, waves, body, opts, keep) structs of a workload dict; keep
    holds the wave arrays the Waves struct points to."""
    g = Grid(cfg["nx"], cfg["ny"], cfg["lx"], cfg["ly"], cfg["depth"])
    f = Fluids(cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"], cfg["g"])
    amp, om, ph = wave_components(cfg["wave"])
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (amp, om, ph)]
    w = Waves(len(amp), _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), cfg["damp_x0"], cfg["damp_len"],
              cfg["probe_x"])
    b = cfg.get("body")
    body = Body(1, b["xc"], b["yc"], b["width"], b["height"], b["mass"], b["added_mass"], b["kappa_p"],
                b["pto_damping"]) if b else Body(0)
    return g, f, w, body, solver_opts(cfg["solver"], precision), keep


class Tank:
    """A 2D wave tank on the GPU (wec_tank_create ... wec_tank_destroy).
    handle: wrap a tank owned by a batch (borrowed; not destroyed here)."""

    def __init__(self, cfg, precision=None, stream=None, handle=None):
        L = load()
        self.cfg = cfg
        self.nx, self.ny = cfg["nx"], cfg["ny"]
        if handle is not None:
            self.h, self.owned = handle, False
            return
        g, f, w, body, o, self._w = tank_structs(cfg, precision)
        h = C.c_void_p()
        _check(L.wec_tank_create(C.byref(g), C.byref(f), C.byref(w), C.byref(body), C.byref(o),
                                 _stream(stream), C.byref(h)))
        self.h, self.owned = h, True

    def close(self):
        if getattr(self, "h", None):
            if self.owned:
                load().wec_tank_destroy(self.h)
            self.h = None

    __del__ = close

    def mg_tiles(self):
        tx, ty, nl = (C.c_int * 32)(), (C.c_int * 32)(), C.c_int(0)
        _check(load().wec_tank_mg_tiles(self.h, tx, ty, 32, C.byref(nl)))
        return [(tx[k], ty[k]) for k in range(max(nl.value - 1, 0))]

    def use_graph(self, enable=True):
        _check(load().wec_tank_use_graph(self.h, 1 if enable else 0))

    def shape(self, f):
        f = FIELD_NAMES.get(f, f)
        if f in (F_U, F_USTAR, F_BETA_U):
            return (self.ny, self.nx + 1)
        if f in (F_V, F_VSTAR, F_BETA_V):
            return (self.ny + 1, self.nx)
        return (self.ny, self.nx)

    def get(self, f):
        f = FIELD_NAMES.get(f, f)
        a = np.zeros(self.shape(f))
        _check(load().wec_get_field(self.h, f, _ptr(a), a.size))
        return a

    def set(self, f, a):
        f = FIELD_NAMES.get(f, f)
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shape(f):
            raise ValueError(f"shape {a.shape} != {self.shape(f)}")
        _check(load().wec_set_field(self.h, f, _ptr(a), a.size))

    def state(self):
        a = np.zeros(5)
        _check(load().wec_get_state(self.h, _ptr(a)))
        return dict(t=a[0], yc=a[1], zdot=a[2], zdot_prev=a[3], yc0=a[4])

    def set_state(self, t, yc, zdot, zdot_prev=None):
        _check(load().wec_set_state(self.h, t, yc, zdot, zdot if zdot_prev is None else zdot_prev))

    def step(self, dt, f_pto=0.0, allow=(WEC_OK, WEC_ERR_NOT_CONVERGED)):
        r = StepResult()
        _check(load().wec_step(self.h, dt, f_pto, C.byref(r)), ok=allow)
        return r.as_dict()

    def step_n(self, n, dt, pto=None, records=True):
        out = (StepResult * n)() if records else None
        p = None if pto is None else _ptr(np.ascontiguousarray(pto, dtype=np.float64))
        _check(load().wec_step_n(self.h, n, dt, p, out))
        return [r.as_dict() for r in out] if records else None

    def set_net(self, net):
        self._net = net  # keep it alive while set
        _check(load().wec_tank_set_net(self.h, None if net is None else net.h))

    def net_stats(self):
        a, b = C.c_longlong(0), C.c_longlong(0)
        _check(load().wec_tank_net_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def pressure_solve(self, rhs, p, rtol):
        it = C.c_int(0)
        rr = C.c_double(0)
        code = _check(load().wec_pressure_solve(self.h, _dev(rhs), _dev(p), rtol, C.byref(it), C.byref(rr)),
                      ok=(WEC_OK, WEC_ERR_NOT_CONVERGED))
        return dict(iters=it.value, relres=rr.value, status=code)

    def save(self):
        n = C.c_size_t(0)
        _check(load().wec_save(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().wec_save(self.h, buf, C.byref(n)))
        return buf.raw

    def load_state(self, data):
        buf = C.create_string_buffer(data, len(data))
        _check(load().wec_load(self.h, buf, len(data)))


def set_option(name, value):
    _check(load().wec_set_option(name.encode(), int(value)))


def launch_count():
    return load().wec_launch_count()


def check_conversions(values):
    """Values (a contiguous FP64 CUDA tensor) for which the library's
    integer-pipe float <-> double conversions differ in any bit from the
    conversion instructions (wec_check_conversions)."""
    import torch
    bad = torch.zeros(1, dtype=torch.int64, device=values.device)
    stream = C.c_void_p(torch.cuda.current_stream(values.device).cuda_stream)
    _check(load().wec_check_conversions(values.numel(), C.c_void_p(values.data_ptr()), C.c_void_p(bad.data_ptr()),
                                        stream))
    return int(bad.item())


def profile_enable(mode, only=None):
    _check(load().wec_profile_enable(mode, only.encode() if only else None))


def profile_read():
    """Aggregated per-(kernel, level) timings since the last read."""
    mx, stride = 256, 64
    names = C.create_string_buffer(mx * stride)
    lv = (C.c_int * mx)()
    la = (C.c_longlong * mx)()
    ms = (C.c_double * mx)()
    by = (C.c_double * mx)()
    cnt = C.c_int(0)
    _check(load().wec_profile_read(mx, names, stride, lv, la, ms, by, C.byref(cnt)))
    out = []
    for k in range(min(cnt.value, mx)):
        nm = names.raw[k * stride:(k + 1) * stride].split(b"\0")[0].decode()
        out.append(dict(name=nm, level=lv[k], launches=la[k], ms=ms[k], bytes=by[k]))
    return out


class Nlfk:
    """Static-grid non-linear Froude-Krylov force (wec_nlfk_create ... destroy).
    region = (x0, y0, h, nx, ny); body = dict(xc, width, height); waves: arrays
    (amp, omega, phase).  force(t, yc, mode) -> (fx, fy) per unit span; mode 0
    incident-wave pressure, 1 hydrostatic (nonlinear buoyancy)."""

    def __init__(self, region, depth, amp, omega, phase, body, rho_w=1025.0, g=9.81, stream=None):
        self._w = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (amp, omega, phase)]
        w = Waves(len(self._w[0]), _ptr(self._w[0]), _ptr(self._w[1]), _ptr(self._w[2]), 0.0, 0.0, 0.0)
        f = Fluids(rho_w, 1.225, 1e-3, 1.8e-5, g)
        bd = Body(1, body["xc"], 0.0, body["width"], body["height"], 1.0, 0.0, 1e-8, 0.0)
        R = Region(*region)
        h = C.c_void_p()
        _check(load().wec_nlfk_create(C.byref(R), C.byref(f), depth, C.byref(w), C.byref(bd), _stream(stream),
                                      C.byref(h)))
        self.h = h

    def force(self, t, yc, mode=0):
        fx, fy = C.c_double(0), C.c_double(0)
        _check(load().wec_nlfk_force(self.h, t, yc, mode, C.byref(fx), C.byref(fy)))
        return fx.value, fy.value

    def close(self):
        if getattr(self, "h", None):
            load().wec_nlfk_destroy(self.h)
            self.h = None

    __del__ = close


# The U-Net's layers (kind, input channels, output channels, level of the
# output), in the parameter order of wec.h; "head" is the 1x1 FP32 output layer.
NET_LAYERS = [("conv3", 2, 32, 0), ("conv3", 32, 32, 0),
              ("down2", 32, 64, 1), ("conv3", 64, 64, 1), ("conv3", 64, 64, 1),
              ("down2", 64, 128, 2), ("conv3", 128, 128, 2), ("conv3", 128, 128, 2),
              ("down2", 128, 256, 3), ("conv3", 256, 256, 3), ("conv3", 256, 256, 3),
              ("up3", 256, 128, 2), ("conv3", 256, 128, 2), ("conv3", 128, 128, 2),
              ("up3", 128, 64, 1), ("conv3", 128, 64, 1), ("conv3", 64, 64, 1),
              ("up3", 64, 32, 0), ("conv3", 64, 32, 0), ("conv3", 32, 32, 0),
              ("head", 32, 1, 0)]


def net_param_shapes():
    """Shapes of the parameter tensors (weights, then bias, per layer)."""
    out = []
    for kind, ci, co, _ in NET_LAYERS:
        w = (ci, co) if kind == "head" else ((2, 2, ci, co) if kind == "down2" else (3, 3, ci, co))
        out += [w, (co,)]
    return out


def net_layer_flops(H, W, batch=1):
    """Multiply-add FLOPs (2 per MAC) of each layer's forward convolution."""
    out = []
    for kind, ci, co, lev in NET_LAYERS:
        px = batch * (H >> lev) * (W >> lev)
        taps = 1 if kind == "head" else (4 if kind == "down2" else 9)
        out.append(2.0 * px * taps * ci * co)
    return out


class Net:
    """The learned warm start's U-Net (wec_net_create ... wec_net_destroy).
    Inputs and targets are float32 CUDA tensors: x [batch, H, W, 2], target and
    output [batch, H, W]; parameters are host float32 vectors."""

    def __init__(self, H, W, max_batch=1, stream=None):
        h = C.c_void_p()
        _check(load().wec_net_create(H, W, max_batch, _stream(stream), C.byref(h)))
        self.h, self.H, self.W, self.max_batch = h, H, W, max_batch
        self.n = int(load().wec_net_param_count())

    def close(self):
        if getattr(self, "h", None):
            load().wec_net_destroy(self.h)
            self.h = None

    __del__ = close

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load().wec_net_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))

    def _get(self, fn):
        a = np.empty(self.n, dtype=np.float32)
        _check(fn(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))
        return a

    def params(self):
        return self._get(load().wec_net_get_params)

    def grads(self):
        return self._get(load().wec_net_get_grads)

    def activation(self, layer, batch, shape):
        """Layer output of the last forward pass as float32 [batch, h, w, c]
        (the library's chunk-planar [batch, h, c / 8, w, 8] reordered)."""
        n, h, w, c = shape
        a = np.empty(int(np.prod(shape)), dtype=np.uint16)
        _check(load().wec_net_get_activation(self.h, layer, batch, a.ctypes.data_as(C.POINTER(C.c_uint16)), a.size))
        f = (a.astype(np.uint32) << 16).view(np.float32).reshape(n, h, c // 8, w, 8)
        return np.ascontiguousarray(f.transpose(0, 1, 3, 2, 4).reshape(n, h, w, c))

    def forward(self, x, out):
        _check(load().wec_net_forward(self.h, x.shape[0], _dev32(x), _dev32(out)))

    def loss_grad(self, x, target):
        loss = C.c_double(0)
        _check(load().wec_net_loss_grad(self.h, x.shape[0], _dev32(x), _dev32(target), C.byref(loss)))
        return loss.value

    def adam(self, lr):
        _check(load().wec_net_adam(self.h, lr))

    def train_step(self, xs, ts, idx, lr):
        i = np.ascontiguousarray(idx, dtype=np.int32)
        loss = C.c_double(0)
        _check(load().wec_net_train_step(self.h, _dev32(xs), _dev32(ts), i.ctypes.data_as(C.POINTER(C.c_int)),
                                         i.size, lr, C.byref(loss)))
        return loss.value


def net_sample(tank, x, t):
    """Features x [ny, nx, 2] and target t [ny, nx] (float32 CUDA tensors) of the
    tank's last pressure problem."""
    _check(load().wec_net_sample(tank.h, _dev32(x), _dev32(t)))


class Batch:
    """Tanks stepping together, one graph launch per batch step
    (wec_batch_create ... wec_batch_destroy)."""

    def __init__(self, cfgs, precision=None, stream=None):
        L = load()
        self.cfgs = list(cfgs)
        n = len(self.cfgs)
        st = [tank_structs(c, precision) for c in self.cfgs]
        self._keep = [x[5] for x in st]
        arrs = [(T * n)(*[x[k] for x in st]) for k, T in enumerate((Grid, Fluids, Waves, Body, SolverOpts))]
        h = C.c_void_p()
        _check(L.wec_batch_create(n, *arrs, _stream(stream), C.byref(h)))
        self.h = h
        self.tanks = []
        for i, c in enumerate(self.cfgs):
            th = C.c_void_p()
            _check(L.wec_batch_tank(h, i, C.byref(th)))
            self.tanks.append(Tank(c, handle=th))

    def __len__(self):
        return len(self.cfgs)

    def close(self):
        if getattr(self, "h", None):
            for t in self.tanks:
                t.h = None
            load().wec_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def step(self, dt, pto=None, allow=(WEC_OK, WEC_ERR_NOT_CONVERGED)):
        n = len(self)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        p = None if pto is None else np.ascontiguousarray(np.broadcast_to(np.asarray(pto, np.float64), (n,)))
        out = (StepResult * n)()
        _check(load().wec_batch_step(self.h, _ptr(d), None if p is None else _ptr(p), out), ok=allow)
        return [r.as_dict() for r in out]

    def step_n(self, nsteps, dt, pto=None, records=True):
        n = len(self)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (nsteps, n)))
        p = None if pto is None else np.ascontiguousarray(np.broadcast_to(np.asarray(pto, np.float64),
                                                                               (nsteps, n)))
        out = (StepResult * (nsteps * n))() if records else None
        _check(load().wec_batch_step_n(self.h, nsteps, _ptr(d), None if p is None else _ptr(p), out),
               ok=(WEC_OK, WEC_ERR_NOT_CONVERGED))
        return [r.as_dict() for r in out] if records else None


class Poisson:
    """Standalone pressure operator and solver on caller coefficients (torch CUDA tensors)."""

    def __init__(self, nx, ny, precision=PREC_FP64, restart=20, mg_pre=2, mg_post=2, stream=None):
        o = SolverOpts(precision, 1e-8, 1000, restart, 0, 1, mg_pre, mg_post)
        h = C.c_void_p()
        _check(load().wec_poisson_create(nx, ny, C.byref(o), _stream(stream), C.byref(h)))
        self.h, self.nx, self.ny = h, nx, ny

    def close(self):
        if getattr(self, "h", None):
            load().wec_poisson_destroy(self.h)
            self.h = None

    __del__ = close

    def set_coefficients(self, bu, bv):
        _check(load().wec_poisson_set_coefficients(self.h, _dev(bu), _dev(bv)))

    def apply(self, x, y):
        _check(load().wec_poisson_apply(self.h, _dev(x), _dev(y)))

    def vcycle(self, b, x):
        _check(load().wec_poisson_vcycle(self.h, _dev(b), _dev(x)))

    def solve(self, b, x, rtol=1e-10, max_iters=500):
        it = C.c_int(0)
        rr = C.c_double(0)
        code = _check(load().wec_poisson_solve(self.h, _dev(b), _dev(x), rtol, max_iters, C.byref(it),
                                               C.byref(rr)), ok=(WEC_OK, WEC_ERR_NOT_CONVERGED))
        return dict(iters=it.value, relres=rr.value, status=code)


class Poisson3(Poisson):
    """The 3D pressure operator and solver (wec_poisson_create3) on caller
    coefficients beta_x (nz, ny, nx+1), beta_y (nz, ny+1, nx), beta_z (nz+1,
    ny, nx); vectors (nz, ny, nx); torch CUDA FP64 tensors."""

    def __init__(self, nx, ny, nz, precision=PREC_FP64, restart=20, mg_pre=2, mg_post=2, stream=None):
        o = SolverOpts(precision, 1e-8, 1000, restart, 0, 1, mg_pre, mg_post)
        h = C.c_void_p()
        _check(load().wec_poisson_create3(nx, ny, nz, C.byref(o), _stream(stream), C.byref(h)))
        self.h, self.nx, self.ny, self.nz = h, nx, ny, nz

    def _n(self, *ts):
        n = self.nx * self.ny * self.nz
        for t in ts:
            if t.numel() != n:
                raise ValueError(f"expected {n} cells, got {t.numel()}")

    def set_coefficients(self, bx, by, bz):
        nx, ny, nz = self.nx, self.ny, self.nz
        for t, m in ((bx, (nx + 1) * ny * nz), (by, nx * (ny + 1) * nz), (bz, nx * ny * (nz + 1))):
            if t.numel() != m:
                raise ValueError(f"expected {m} face coefficients, got {t.numel()}")
        _check(load().wec_poisson_set_coefficients3(self.h, _dev(bx), _dev(by), _dev(bz)))

    def apply(self, x, y):
        self._n(x, y)
        super().apply(x, y)

    def vcycle(self, b, x):
        self._n(b, x)
        super().vcycle(b, x)

    def solve(self, b, x, rtol=1e-10, max_iters=500):
        self._n(b, x)
        return super().solve(b, x, rtol, max_iters)


class Tank3:
    """The level-set part of the 3D tank on the GPU (wec_tank3_*): ``cfg`` is a
    3D workload dict (synth.tank3d); fields are numpy FP64 arrays, cells (nz, ny,
    nx), u (nz, ny, nx+1), v (nz, ny+1, nx), w (nz+1, ny, nx)."""

    def __init__(self, cfg, precision=None, stream=None, step=True):
        L = load()
        self.cfg = cfg
        nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
        g = Grid3(nx, ny, nz, cfg["lx"], cfg["ly"], cfg["lz"], cfg["depth"])
        f = Fluids(cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"], cfg["g"])
        amp, om, ph = wave_components(cfg["wave"])
        self._w = [np.ascontiguousarray(a, dtype=np.float64) for a in (amp, om, ph)]
        w = Waves(len(amp), _ptr(self._w[0]), _ptr(self._w[1]), _ptr(self._w[2]), cfg["damp_x0"], cfg["damp_len"],
                  cfg["probe_x"])
        b = cfg.get("body")
        body = Cylinder(1, b["xc"], b["yc"], b["radius"], b["length"], b["mass"], b["zc"], b["kappa_p"],
                        b["added_mass"], b.get("pto_damping", 0.0)) if b else Cylinder(0)
        o = solver_opts(cfg["solver"], precision) if step else None
        h = C.c_void_p()
        _check(L.wec_tank3_create(C.byref(g), C.byref(f), C.byref(w), C.byref(body), C.byref(o) if o else None,
                                  _stream(stream), C.byref(h)))
        self.h = h
        self.shapes = {F3_SIGMA: (nz, ny, nx), F3_U: (nz, ny, nx + 1), F3_V: (nz, ny + 1, nx),
                       F3_W: (nz + 1, ny, nx)}
        for fid in (F3_RHO, F3_MU, F3_RHO_FLOW, F3_CHI, F3_P):
            self.shapes[fid] = (nz, ny, nx)

    def close(self):
        if getattr(self, "h", None):
            load().wec_tank3_destroy(self.h)
            self.h = None

    __del__ = close

    def get(self, fid):
        a = np.zeros(self.shapes[fid])
        _check(load().wec_tank3_get_field(self.h, fid, _ptr(a), a.size))
        return a

    def set(self, fid, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shapes[fid]:
            raise ValueError(f"expected shape {self.shapes[fid]}, got {a.shape}")
        _check(load().wec_tank3_set_field(self.h, fid, _ptr(a), a.size))

    def materials(self, zc):
        _check(load().wec_tank3_materials(self.h, zc))
        return {k: self.get(f) for k, f in (("rho", F3_RHO), ("mu", F3_MU), ("rho_flow", F3_RHO_FLOW),
                                            ("chi", F3_CHI))}

    def advect(self, dt, t):
        _check(load().wec_tank3_advect(self.h, dt, t))

    def reinit(self, nit, t):
        _check(load().wec_tank3_reinit(self.h, nit, t))

    def step(self, dt, pto=0.0):
        r = StepResult()
        code = _check(load().wec_tank3_step(self.h, dt, pto, C.byref(r)), ok=(WEC_OK, WEC_ERR_NOT_CONVERGED))
        d = r.as_dict()
        d["status"] = code
        return d

    def state(self):
        a = np.zeros(5)
        _check(load().wec_tank3_get_state(self.h, _ptr(a)))
        return dict(t=a[0], zc=a[1], zdot=a[2], zc0=a[3], zdot_prev=a[4])
