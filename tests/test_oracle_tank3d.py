"""Pins of the 3D tank-step oracle (the step of sections "Continuous equations
of motion" through "Fluid-structure coupling" with d = 3).  None of the
expected values comes from the CUDA library.

- reduction: with no body, a state constant along y with v = 0 steps as the 2D
  oracle's step (which has pins of its own), boundaries, inflow, damping zone
  and pressure solve included (to the solver tolerance: the 3D multigrid
  differs);
- still water without a body stays at rest (hydrostatic balance on the MAC grid);
- the projected velocity is divergence-free to the solver tolerance
  (||h div u|| = ||b - A phi|| <= rtol ||b||);
- the heave force on the floating cylinder in hydrostatic water is its weight
  (Archimedes), to the accuracy of the voxelised bottom area;
- the Brinkman term holds the body's fluid at its heave velocity.
"""
import math

import numpy as np
import pytest

from oracle import tank as O2
from oracle import tank3d as T3
from paper_2206_07732_gb300 import synth


def _cfg(nx=32, ny=8, nz=16, body=False, rtol=1e-12, **kw):
    c = synth.tank3d(seed=5, nx=nx, ny=ny, nz=nz, rtol=rtol, **kw)
    if not body:
        c["body"] = None
    return c


def _cfg2(c3):
    c2 = dict(c3)
    c2["ny"], c2["ly"], c2["body"] = c3["nz"], c3["lz"], None
    return c2


def test_y_invariant_step_is_the_2d_step():
    c = _cfg()
    t3, t2 = T3.OracleTank3(c), O2.OracleTank(_cfg2(c))
    # the two oracles' initial states are the same construction
    s2, u2, w2, p2 = t2.get(O2.F_SIGMA), t2.get(O2.F_U), t2.get(O2.F_V), t2.get(O2.F_P)
    for a3, a2 in ((t3.get(T3.F_SIGMA), s2), (t3.get(T3.F_U), u2), (t3.get(T3.F_W), w2), (t3.get(T3.F_P), p2)):
        for j in range(c["ny"]):
            assert np.array_equal(a3[:, j, :], a2)
    for _ in range(3):
        r3, r2 = t3.step(c["dt"]), t2.step(c["dt"])
        assert r3["status"] == 0 and r2["status"] == 0
    for f3, f2 in ((T3.F_SIGMA, O2.F_SIGMA), (T3.F_U, O2.F_U), (T3.F_W, O2.F_V), (T3.F_P, O2.F_P)):
        a3, a2 = t3.get(f3), t2.get(f2)
        err = max(np.max(np.abs(a3[:, j, :] - a2)) for j in range(c["ny"])) / np.max(np.abs(a2))
        assert err < 1e-8, (f3, err)
    assert np.max(np.abs(t3.get(T3.F_V))) < 1e-12 * np.max(np.abs(t3.get(T3.F_U)))
    assert r3["eta_probe"] == pytest.approx(r2["eta_probe"], rel=1e-8)


def test_still_water_stays_at_rest():
    c = _cfg(nx=16, ny=8, nz=16)
    c["wave"] = dict(kind="regular", H=0.0, T=1.0, phase=0.0)
    t = T3.OracleTank3(c)
    for _ in range(5):
        assert t.step(c["dt"])["status"] == 0
    for f in (T3.F_U, T3.F_V, T3.F_W):
        assert np.max(np.abs(t.get(f))) < 1e-10


def test_divergence_below_solver_tolerance():
    c = _cfg(nx=32, ny=8, nz=16, body=True, rtol=1e-8)
    t = T3.OracleTank3(c)
    for _ in range(3):
        r = t.step(c["dt"])
    u, v, w = t.get(T3.F_U), t.get(T3.F_V), t.get(T3.F_W)
    h = c["lx"] / c["nx"]
    div = h * ((u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :]) + (w[1:] - w[:-1]))
    assert np.linalg.norm(div) == pytest.approx(r["div_norm"], rel=1e-6)
    assert r["div_norm"] <= 1.01 * c["solver"]["rtol"] * r["rhs_norm"]
    assert r["div_norm"] == pytest.approx(r["residual"] * r["rhs_norm"], rel=1e-3)


def _cylinder_box(h=1.0 / 16):
    # a 2 m x 2 m x 4 m tank around the cylinder (R / h = 8), still water
    n = int(round(2.0 / h))
    c = synth.tank3d(seed=0, nx=n, ny=n, nz=2 * n, rtol=1e-10)
    c["lx"], c["ly"], c["lz"] = 2.0, 2.0, 4.0
    c["wave"] = dict(kind="regular", H=0.0, T=1.0, phase=0.0)
    c["damp_len"] = 0.0
    c["body"] = synth.cylinder_body(1.0, 1.0, 0.5, 0.8, 0.4, 2.0, c["rho_w"])
    return c


def test_floating_cylinder_force_is_its_weight():
    c = _cylinder_box()
    t = T3.OracleTank3(c)
    b = c["body"]
    F = t.force()
    print(f"F = {F:.2f} N, m g = {b['mass'] * c['g']:.2f} N")
    assert F == pytest.approx(b["mass"] * c["g"], rel=0.03)


def test_brinkman_holds_the_body_fluid_at_its_heave_velocity():
    c = _cylinder_box(h=1.0 / 8)
    c["body"]["zc"] -= 0.05  # released 5 cm deep: it rises
    t = T3.OracleTank3(c)
    for _ in range(4):
        t.step(c["dt"])
    zd = t.body()["zdot"]
    assert zd > 0.0
    w = t.get(T3.F_W)
    h = c["lx"] / c["nx"]
    b = c["body"]
    zc = t.body()["zc"]
    i0, i1 = int((b["xc"] - 0.3) / h), int((b["xc"] + 0.3) / h)
    k0, k1 = int((zc - 0.3) / h), int((zc + 0.3) / h)
    # z-faces well inside the cylinder: w -> zdot, u and v -> 0, to the
    # penalisation's own accuracy O(rho kappa_p / dt) (~1 % here) while the body
    # accelerates; the 2D pin uses the same 5 % bound
    scale = max(abs(zd), 1e-3)
    assert np.max(np.abs(w[k0:k1, i0:i1, i0:i1] - zd)) < 0.05 * scale
    assert np.max(np.abs(t.get(T3.F_U)[k0:k1, i0:i1, i0:i1])) < 0.05 * scale
    assert np.max(np.abs(t.get(T3.F_V)[k0:k1, i0:i1, i0:i1])) < 0.05 * scale
