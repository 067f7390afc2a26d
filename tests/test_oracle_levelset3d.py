"""Pins of the 3D level-set oracle (advection, reinitialisation, materials of
the 3D tank; sections "Interface tracking", "Level set advection", "Density and
viscosity specification" with d = 3).  None of the expected values comes from
the CUDA library.

- reduction: a field constant along y with v = 0 is advected, reinitialised
  and given materials exactly as the 2D oracle (which has pins of its own) does
  in the (x, vertical) plane, boundaries included;
- closed forms: PPM transports a linear field exactly (interior cells), a
  constant stays constant; reinitialisation restores |grad sigma| = 1 around a
  sphere without moving it; the cylinder's material fields give its volume and
  mass.
"""
import math

import numpy as np
import pytest

from oracle import levelset3d as L3
from oracle import tank as O2
from oracle import waves as W
from paper_2206_07732_gb300 import synth


def _cfg(nx=32, ny=8, nz=16, body=False, damp=True):
    c = synth.tank3d(seed=3, nx=nx, ny=ny, nz=nz)
    if not body:
        c["body"] = None
    if not damp:
        c["damp_len"] = 0.0
    return c


def _cfg2(c3):
    c2 = dict(c3)
    c2["ny"], c2["ly"], c2["body"] = c3["nz"], c3["lz"], None
    return c2


def _surface_sigma(c, noise_seed=0):
    # sigma = z - depth - eta(x, 0) plus a smooth perturbation, in the (x, z) plane
    nx, nz, h = c["nx"], c["nz"], c["lx"] / c["nx"]
    amp, om, k, ph = W.components(c["wave"], c["depth"], c["g"])
    x = (np.arange(nx) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    eta = np.sum(amp[:, None] * np.cos(k[:, None] * x[None, :] + ph[:, None]), axis=0)
    rng = np.random.default_rng(noise_seed)
    pert = 0.05 * np.sin(2 * np.pi * x[None, :] / 3.0 + rng.uniform()) * np.cos(np.pi * z[:, None] / 2.0)
    return z[:, None] - c["depth"] - eta[None, :] + pert


def _y_invariant_case(c):
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    s2 = _surface_sigma(c)
    rng = np.random.default_rng(5)
    u2 = 0.4 * rng.standard_normal((nz, nx + 1))
    w2 = 0.4 * rng.standard_normal((nz + 1, nx))
    s3 = np.repeat(s2[:, None, :], ny, axis=1)
    u3 = np.repeat(u2[:, None, :], ny, axis=1)
    v3 = np.zeros((nz, ny + 1, nx))
    w3 = np.repeat(w2[:, None, :], ny, axis=1)
    return (s2, u2, w2), (s3, u3, v3, w3)


def test_y_invariant_advection_is_the_2d_advection():
    c = _cfg()
    (s2, u2, w2), (s3, u3, v3, w3) = _y_invariant_case(c)
    o3 = L3.Oracle3(c)
    out3 = o3.advect(s3, u3, v3, w3, 0.02, 0.0)
    t2 = O2.OracleTank(_cfg2(c))
    t2.set(O2.F_SIGMA, s2)
    t2.set(O2.F_U, u2)
    t2.set(O2.F_V, w2)
    t2.advect(0.02)
    out2 = t2.get(O2.F_SIGMA)
    for j in range(c["ny"]):
        assert np.array_equal(out3[:, j, :], out2), j


def test_y_invariant_reinitialisation_is_the_2d_one():
    c = _cfg()
    (s2, _, _), (s3, _, _, _) = _y_invariant_case(c)
    s2 = 1.7 * s2  # not a distance: reinitialisation has work to do
    s3 = 1.7 * s3
    out3 = L3.Oracle3(c).reinit(s3, 4, 0.0)
    t2 = O2.OracleTank(_cfg2(c))
    t2.set(O2.F_SIGMA, s2)
    t2.reinit(4)
    out2 = t2.get(O2.F_SIGMA)
    for j in range(c["ny"]):
        assert np.array_equal(out3[:, j, :], out2), j


def test_y_invariant_materials_are_the_2d_ones():
    c = _cfg()
    (s2, _, _), (s3, _, _, _) = _y_invariant_case(c)
    m3 = L3.Oracle3(c).materials(s3, 0.0)
    t2 = O2.OracleTank(_cfg2(c))
    t2.set(O2.F_SIGMA, s2)
    m2 = t2.materials()
    for key in ("rho", "mu", "rho_flow", "chi"):
        for j in range(c["ny"]):
            assert np.array_equal(m3[key][:, j, :], m2[key]), key


@pytest.mark.parametrize("grad,vel", [((0.0, 0.2, 1.0), (0.0, 0.3, 0.0)), ((0.1, -0.3, 1.0), (0.2, -0.1, 0.15))])
def test_linear_field_is_transported_exactly(grad, vel):
    # uniform velocity, sigma linear: the PPM faces reproduce it, so interior
    # cells (3 or more from every boundary) move by -dt (vel . grad)
    c = _cfg(nx=24, ny=16, nz=16, damp=False)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    h = c["lx"] / nx
    x, y, z = ((np.arange(m) + 0.5) * h for m in (nx, ny, nz))
    s = grad[0] * x[None, None, :] + grad[1] * y[None, :, None] + grad[2] * (z[:, None, None] - c["depth"])
    u = np.full((nz, ny, nx + 1), vel[0])
    v = np.full((nz, ny + 1, nx), vel[1])
    w = np.full((nz + 1, ny, nx), vel[2])
    dt = 0.05
    out = L3.Oracle3(c).advect(s, u, v, w, dt, 0.0)
    expect = s - dt * (vel[0] * grad[0] + vel[1] * grad[1] + vel[2] * grad[2])
    sl = (slice(3, nz - 3), slice(3, ny - 3), slice(3, nx - 3))
    assert np.max(np.abs(out[sl] - expect[sl])) < 1e-13


def test_constant_field_stays_constant():
    c = _cfg(nx=16, ny=8, nz=8, damp=False)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    f = synth.random_fields3(nx, ny, nz, seed=2, scale=0.5)
    s = np.full((nz, ny, nx), 0.37)
    out = L3.Oracle3(c).advect(s, f["u"], f["v"], f["w"], 0.01, 0.0)
    assert np.max(np.abs(out[:, :, 3:] - 0.37)) < 1e-15  # columns 0-2 see the inflow ghost


def test_reinitialisation_restores_a_sphere_distance():
    c = _cfg(nx=40, ny=40, nz=40, damp=False)
    c["lx"] = 2.0  # h = 0.05
    h = c["lx"] / c["nx"]
    x = (np.arange(40) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R, x0 = 0.5, 1.0
    r = np.sqrt((X - x0) ** 2 + (Y - x0) ** 2 + (Z - x0) ** 2)
    s0 = (r - R) * (1.0 + 0.8 * (r - R))  # right zero set, wrong slope (0.2 .. 1.8)
    c["depth"] = 1.0  # (ghosts are not reached near the sphere)
    s = L3.Oracle3(c).reinit(s0, 40, 0.0)
    band = np.abs(r - R) < 2.5 * h
    gz, gy, gx = np.gradient(s, h)
    gn = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)[band]
    assert np.mean(np.abs(gn - 1.0)) < 0.05
    # the zero set stays: near-interface cells keep their sign and sigma ~ r - R
    near = np.abs(r - R) < 0.5 * h
    assert np.max(np.abs(s[near] - (r - R)[near])) < 0.25 * h


def test_cylinder_materials_give_its_volume_and_mass():
    c = _cfg(nx=64, ny=32, nz=32, body=True)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    h = c["lx"] / nx
    b = c["body"]
    s = np.full((nz, ny, nx), -10.0)  # all water (sigma below the band)
    m = L3.Oracle3(c).materials(s, b["zc"])
    # chi = 1 - H_body is the body indicator (1 inside, where the Brinkman term acts)
    vol = np.sum(m["chi"]) * h ** 3
    rho_s = b["mass"] / (math.pi * b["radius"] ** 2 * b["length"])
    assert vol == pytest.approx(math.pi * b["radius"] ** 2 * b["length"], rel=0.03)
    # the body's mass: what the density carries beyond the surrounding water's
    # share (1 - chi) rho_w (all fluid is water here), equal to m to the
    # accuracy of the voxelised volume
    assert np.sum(m["rho"] - c["rho_w"] * (1.0 - m["chi"])) * h ** 3 == pytest.approx(b["mass"], rel=0.03)
    x, y, z = ((np.arange(q) + 0.5) * h for q in (nx, ny, nz))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    psi = np.maximum(np.hypot(X - b["xc"], Y - b["yc"]) - b["radius"], np.abs(Z - b["zc"]) - 0.5 * b["length"])
    deep, out = psi < -h, psi > h
    assert np.allclose(m["rho"][deep], rho_s) and np.all(m["chi"][deep] == 1.0)
    assert np.all(m["mu"][deep] == c["mu_w"])
    assert np.all(m["chi"][out] == 0.0) and np.all(m["rho"][out] == c["rho_w"])
    assert np.all(m["rho_flow"] == c["rho_w"])
