"""Pins of the 3D oracle's fixed-point cycles (section "Time stepping scheme":
n_cycles cycles per step; cycle k evaluates the force on the iterate
(p, u, z)^{n+1,k}, updates the heave from level n, advects sigma^n with the
means of levels n and n+1,k, and solves level n's momentum system with the
iterate's pressure and body velocity; one cycle is the plain step)."""
import math

import numpy as np
import pytest

from oracle import levelset3d as L3
from oracle import tank3d as T3
from paper_2206_07732_gb300 import synth


def _cfg(n_cycles, seed=1, shape=(32, 8, 16), body=True):
    c = synth.tank3d(seed=seed, nx=shape[0], ny=shape[1], nz=shape[2], rtol=1e-12)
    c["solver"]["n_cycles"] = n_cycles
    if not body:
        c["body"] = None
    return c


def test_cycle_advection_is_exact_on_linear_fields():
    # base sigma^n and the mean field linear, velocities uniform: the cycle's
    # update is sigma^n - dt (u_mean . grad sigma_mean) exactly (PPM is exact on
    # linear fields); a base / field mix-up or a missing mean fails it
    c = _cfg(2, body=False)
    c["damp_len"] = 0.0
    O = L3.Oracle3(c)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    h = c["lx"] / nx
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                          indexing="ij")
    sig_n = 0.3 * x - 0.2 * y + 0.7 * z - 1.1
    sig_k = sig_n + (0.1 * x + 0.05 * y - 0.2 * z + 0.01)
    mean = 0.5 * (sig_n + sig_k)
    un, uk = (0.2, -0.1, 0.15), (0.4, 0.1, -0.05)
    um = [0.5 * (a + b) for a, b in zip(un, uk)]
    U = np.full((nz, ny, nx + 1), um[0])
    V = np.full((nz, ny + 1, nx), um[1])
    W = np.full((nz + 1, ny, nx), um[2])
    dt = 2e-3
    out = O.advect_half(sig_n, mean, U, V, W, dt, 0.0, dt)
    grad = (0.3 + 0.05, -0.2 + 0.025, 0.7 - 0.1)  # gradient of the mean field
    want = sig_n - dt * (um[0] * grad[0] + um[1] * grad[1] + um[2] * grad[2])
    sl = (slice(3, -3), slice(3, -3), slice(3, -3))
    np.testing.assert_allclose(out[sl], want[sl], rtol=0, atol=1e-13)


def test_one_cycle_is_the_plain_step():
    a, b = T3.OracleTank3(_cfg(1)), T3.OracleTank3(_cfg(0))
    for _ in range(2):
        ra, rb = a.step(1e-3), b.step(1e-3)
    for f in range(5):
        assert np.array_equal(a.get(f), b.get(f))
    assert ra["zdot"] == rb["zdot"]


def test_second_cycle_takes_the_force_of_the_first_iterate_and_the_heave_from_level_n():
    dt = 1e-3
    c1, c2 = _cfg(1), _cfg(2)
    a = T3.OracleTank3(c1)
    a.step(dt)
    F1 = a.force()  # the force on the first cycle's iterate (p, u, z)^{n+1,1}
    b = T3.OracleTank3(c2)
    r = b.step(dt)
    assert r["f_hydro"] == F1
    # Eq. newton_u with the stabilising mass of the heave update, from level n
    # (zdot^n = zdot^{n-1} = 0 at creation)
    bd = c2["body"]
    m, ma, g = bd["mass"], bd["added_mass"], c2["g"]
    zd = (dt * (F1 - m * g)) / (m + ma)
    assert r["zdot"] == pytest.approx(zd, rel=1e-14, abs=1e-18)


def test_cycles_keep_still_water_at_rest():
    c = _cfg(2, body=False)
    c["wave"] = {"kind": "regular", "H": 0.0, "T": 2.0, "phase": 0.0}
    o = T3.OracleTank3(c)
    for _ in range(5):
        o.step(1e-3)
    assert max(float(np.max(np.abs(o.get(f)))) for f in (T3.F_U, T3.F_V, T3.F_W)) < 1e-10


def test_cycles_converge_to_a_fixed_point():
    # one step from the same state with 1, 2, 3, 4 cycles: successive
    # differences shrink (a contraction), the first one is not zero.  The
    # iteration on the force coupling contracts by about m_added / (m + m_a): with
    # the stabilising mass rho_w pi R^2 L (twice the body's) quickly; without it
    # (the cylinder's added mass ~0.9 of its mass) slowly
    us = []
    for nc in (1, 2, 3, 4):
        c = _cfg(nc, seed=5)
        b = c["body"]
        b["added_mass"] = c["rho_w"] * math.pi * b["radius"] ** 2 * b["length"]
        o = T3.OracleTank3(c)
        r = o.step(2e-3)
        us.append((o.get(T3.F_U), o.get(T3.F_W), r["zdot"]))
    d = [max(float(np.max(np.abs(us[k + 1][0] - us[k][0]))), float(np.max(np.abs(us[k + 1][1] - us[k][1]))))
         for k in range(3)]
    print("cycle differences", d)
    assert d[0] > 0.0
    assert d[1] < 0.5 * d[0] and d[2] < 0.5 * d[1]
