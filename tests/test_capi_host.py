"""CPU-only checks of the C ABI library: it loads, exports every declared symbol,
validates arguments on the host, and its host wave utilities agree with the oracle.
No device compute is called here."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2206_07732_gb300 import build as B
from paper_2206_07732_gb300 import synth
from paper_2206_07732_gb300 import wec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return wec.load()


def _declared():
    names = []
    with open(os.path.join(ROOT, "include", "wec.h")) as f:
        text = f.read()
    for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(wec_\w+)\s*\(", text, flags=re.M):
        names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("wec_tank_create", "wec_step", "wec_pressure_solve", "wec_tank_destroy", "wec_last_error"):
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_targets_sm103a():
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _structs(cfg):
    g = wec.Grid(cfg["nx"], cfg["ny"], cfg["lx"], cfg["ly"], cfg["depth"])
    f = wec.Fluids(cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"], cfg["g"])
    amp = np.array([0.01]); om = np.array([6.0]); ph = np.array([0.0])
    w = wec.Waves(1, wec._ptr(amp), wec._ptr(om), wec._ptr(ph), 3.0, 1.0, 0.5)
    b = cfg["body"]
    body = wec.Body(1, b["xc"], b["yc"], b["width"], b["height"], b["mass"], b["added_mass"], b["kappa_p"], 0.0)
    o = wec.solver_opts(cfg["solver"])
    return g, f, w, body, o, (amp, om, ph)


@pytest.mark.parametrize("bad", ["odd", "nonuniform", "depth", "rho", "restart", "kappa", "omega"])
def test_create_rejects_invalid_arguments_on_host(lib, bad):
    cfg = synth.tank_small(nx=64, ny=32)
    g, f, w, body, o, keep = _structs(cfg)
    if bad == "odd":
        g.nx = 63
    elif bad == "nonuniform":
        g.ly = 2.5
    elif bad == "depth":
        g.depth = 5.0
    elif bad == "rho":
        f.rho_a = -1.0
    elif bad == "restart":
        o.restart = 99
    elif bad == "kappa":
        body.kappa_p = 0.0
    elif bad == "omega":
        keep[1][0] = -1.0
    h = C.c_void_p(123)
    code = lib.wec_tank_create(C.byref(g), C.byref(f), C.byref(w), C.byref(body), C.byref(o), None, C.byref(h))
    assert code == wec.WEC_ERR_INVALID
    assert h.value is None
    assert lib.wec_last_error().decode()


def test_null_handles_are_errors(lib):
    r = wec.StepResult()
    assert lib.wec_step(None, 1e-3, 0.0, C.byref(r)) == wec.WEC_ERR_INVALID
    assert lib.wec_pressure_solve(None, None, None, 1e-8, None, None) == wec.WEC_ERR_INVALID
    lib.wec_tank_destroy(None)
    lib.wec_poisson_destroy(None)


def test_wave_utilities_match_oracle(lib):
    from oracle import waves as W
    for d in (0.5, 1.0, 2.5, 2.0):
        for om in np.linspace(0.5, 25.0, 40):
            k = wec.wave_number(om, d, 9.81)
            assert abs(9.81 * k * math.tanh(k * d) - om * om) <= 1e-13 * om * om
            assert k == pytest.approx(W.dispersion_k(om, d, 9.81), rel=1e-13)
            assert wec.wave_number_fenton_kd(om, d, 9.81) == pytest.approx(W.fenton_kd(om, d, 9.81), rel=1e-13)
    ph = np.zeros(64)
    a, om = wec.jonswap(0.15, 1.6, 3.3, 64)
    a0, om0, _ = W.jonswap_components(0.15, 1.6, 3.3, 64, ph)
    np.testing.assert_allclose(om, om0, rtol=1e-14)
    np.testing.assert_allclose(a, a0, rtol=1e-12)


@pytest.mark.parametrize("bad", ["count", "null", "tank"])
def test_batch_create_rejects_invalid_arguments_on_host(lib, bad):
    cfgs = [synth.tank_small(nx=64, ny=32), synth.tank_small(nx=96, ny=48)]
    st = [_structs(c) for c in cfgs]
    arrs = [(T * 2)(*[x[k] for x in st]) for k, T in enumerate((wec.Grid, wec.Fluids, wec.Waves, wec.Body,
                                                                  wec.SolverOpts))]
    n = 2
    if bad == "count":
        n = 0
    elif bad == "null":
        arrs[3] = None
    elif bad == "tank":
        arrs[0][1].nx = 95  # the second tank is invalid: nothing is left allocated
    h = C.c_void_p(123)
    code = lib.wec_batch_create(n, *arrs, None, C.byref(h))
    assert code == wec.WEC_ERR_INVALID
    assert not h.value
    msg = lib.wec_last_error().decode()
    assert ("tank 1" in msg) if bad == "tank" else ("batch" in msg)


def test_options_are_validated_on_host(lib):
    assert lib.wec_set_option(b"mg_bottom_shift", 9) == wec.WEC_ERR_INVALID
    assert lib.wec_set_option(b"mg_bottom_shift", -2) == wec.WEC_ERR_INVALID
    assert lib.wec_set_option(b"no_such_option", 1) == wec.WEC_ERR_INVALID
    assert lib.wec_set_option(b"mg_bottom_shift", 1) == wec.WEC_OK
    assert lib.wec_set_option(b"mg_bottom_shift", -1) == wec.WEC_OK


@pytest.mark.parametrize("bad", ["region", "depth", "body", "omega"])
def test_nlfk_create_validates_on_host(lib, bad):
    R = wec.Region(0.0, 0.0, 0.01, 100, 50)
    f = wec.Fluids(1025.0, 1.225, 1e-3, 1.8e-5, 9.81)
    amp, om, ph = np.array([0.01]), np.array([5.0]), np.array([0.0])
    w = wec.Waves(1, wec._ptr(amp), wec._ptr(om), wec._ptr(ph), 0.0, 0.0, 0.0)
    b = wec.Body(1, 0.5, 0.25, 0.2, 0.1, 1.0, 0.0, 1e-8, 0.0)
    depth = 0.3
    if bad == "region":
        R.h = 0.0
    elif bad == "depth":
        depth = -1.0
    elif bad == "body":
        b.present = 0
    elif bad == "omega":
        om[0] = 0.0
    h = C.c_void_p(123)
    assert lib.wec_nlfk_create(C.byref(R), C.byref(f), depth, C.byref(w), C.byref(b), None, C.byref(h)) == \
        wec.WEC_ERR_INVALID
    assert not h.value
    assert b"nlfk" in lib.wec_last_error()


def test_net_matches_the_oracle_layout_and_validates_on_host(lib):
    # the parameter vector has the oracle's layout size; bad sizes and NULLs
    # are rejected before any device work
    from oracle import unet as U
    assert lib.wec_net_param_count() == sum(int(np.prod(s)) for s in U.param_shapes(32))
    h = C.c_void_p()
    for H, W, b in ((12, 16, 1), (16, 4, 1), (16, 16, 0), (0, 8, 1), (8192, 8192, 2)):
        assert lib.wec_net_create(H, W, b, None, C.byref(h)) == wec.WEC_ERR_INVALID
        assert not h.value
    assert lib.wec_net_create(16, 16, 1, None, None) == wec.WEC_ERR_INVALID
    assert lib.wec_net_forward(None, 1, None, None) == wec.WEC_ERR_INVALID
    assert lib.wec_net_adam(None, C.c_float(1e-3)) == wec.WEC_ERR_INVALID
    assert lib.wec_tank_set_net(None, None) == wec.WEC_ERR_INVALID
    assert lib.wec_net_sample(None, None, None) == wec.WEC_ERR_INVALID
    lib.wec_net_destroy(None)


def test_binding_layer_table_matches_the_oracle():
    from oracle import unet as U
    assert wec.net_param_shapes() == [tuple(s) for s in U.param_shapes(32)]
    assert [(k if k != "head" else "head", ci, co) for k, ci, co, _ in wec.NET_LAYERS] == \
        [(k, ci, co) for _, k, ci, co in U.layers(32)]


@pytest.mark.parametrize("bad", ["nonuniform", "small", "rho", "precision", "restart", "radius", "kappa"])
def test_tank3_create_rejects_invalid_arguments_on_host(lib, bad):
    cfg = synth.tank3d(nx=16, ny=8, nz=8)
    g = wec.Grid3(cfg["nx"], cfg["ny"], cfg["nz"], cfg["lx"], cfg["ly"], cfg["lz"], cfg["depth"])
    f = wec.Fluids(cfg["rho_w"], cfg["rho_a"], cfg["mu_w"], cfg["mu_a"], cfg["g"])
    amp, om, ph = np.array([0.01]), np.array([3.0]), np.array([0.0])
    w = wec.Waves(1, wec._ptr(amp), wec._ptr(om), wec._ptr(ph), 6.0, 2.0, 1.0)
    b = cfg["body"]
    body = wec.Cylinder(1, b["xc"], b["yc"], b["radius"], b["length"], b["mass"], b["zc"], b["kappa_p"],
                        b["added_mass"], 0.0)
    o = wec.solver_opts(cfg["solver"])
    if bad == "nonuniform":
        g.lz = 2.0 * g.lz
    elif bad == "small":
        g.nz = 2
    elif bad == "rho":
        f.rho_w = 0.0
    elif bad == "precision":
        o.precision = 7
    elif bad == "restart":
        o.restart = 0
    elif bad == "radius":
        body.radius = -0.5
    elif bad == "kappa":
        body.kappa_p = 0.0
    h = C.c_void_p(123)
    code = lib.wec_tank3_create(C.byref(g), C.byref(f), C.byref(w), C.byref(body), C.byref(o), None, C.byref(h))
    assert code == wec.WEC_ERR_INVALID
    assert h.value is None
    assert lib.wec_last_error().decode()
    r = wec.StepResult()
    assert lib.wec_tank3_step(None, 1e-3, 0.0, C.byref(r)) == wec.WEC_ERR_INVALID
    lib.wec_tank3_destroy(None)
