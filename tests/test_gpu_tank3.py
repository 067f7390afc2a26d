"""The level-set part of the 3D tank on the GPU (wec_tank3: materials with the
cylinder, PPM advection with the inflow ghost and the damping zone, Sussman
reinitialisation) against the 3D level-set oracle: element by element on small
grids with ragged thread-block rows, a chain of calls, and the 512 x 256 x 256
tank on sampled cells (every boundary face of the box plus random interior
cells)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import levelset3d as L3  # noqa: E402
from oracle import waves as W  # noqa: E402
from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _state(c, seed):
    # sigma: the incident surface z - depth - eta(x, 0) with a perturbation that
    # varies along y; velocities: smooth random fields of 0.3 m/s
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    h = c["lx"] / nx
    amp, om, k, ph = W.components(c["wave"], c["depth"], c["g"])
    x, y, z = ((np.arange(m) + 0.5) * h for m in (nx, ny, nz))
    eta = np.sum(amp[:, None] * np.cos(k[:, None] * x[None, :] + ph[:, None]), axis=0)
    rng = np.random.default_rng(seed)
    s = (z[:, None, None] - c["depth"] - eta[None, None, :] +
         0.05 * np.sin(2 * np.pi * x[None, None, :] / 3.0 + 1.3 * y[None, :, None] + rng.uniform()))
    f = synth.random_fields3(nx, ny, nz, seed=seed + 1, scale=0.3)
    return s, f["u"], f["v"], f["w"]


CASES = [(40, 12, 20), (130, 6, 16), (16, 20, 12)]


@pytest.mark.parametrize("shape", CASES)
def test_materials_match_oracle(shape):
    nx, ny, nz = shape
    c = synth.tank3d(seed=1, nx=nx, ny=ny, nz=nz)
    s, *_ = _state(c, 3)
    T = wec.Tank3(c, step=False)
    T.set(wec.F3_SIGMA, s)
    zc = c["body"]["zc"] - 0.013
    m = T.materials(zc)
    mo = L3.Oracle3(c).materials(s, zc)
    for key in ("rho", "mu", "rho_flow", "chi"):
        assert rel(m[key], mo[key]) < 1e-13, key
    T.close()


@pytest.mark.parametrize("shape", CASES)
def test_advection_matches_oracle(shape):
    nx, ny, nz = shape
    c = synth.tank3d(seed=2, nx=nx, ny=ny, nz=nz)
    s, u, v, w = _state(c, 5)
    T = wec.Tank3(c, step=False)
    for fid, a in ((wec.F3_SIGMA, s), (wec.F3_U, u), (wec.F3_V, v), (wec.F3_W, w)):
        T.set(fid, a)
    T.advect(0.02, 0.37)
    out = T.get(wec.F3_SIGMA)
    ref = L3.Oracle3(c).advect(s, u, v, w, 0.02, 0.37)
    assert rel(out, ref) < 1e-12
    T.close()


@pytest.mark.parametrize("shape", CASES)
def test_reinitialisation_matches_oracle(shape):
    nx, ny, nz = shape
    c = synth.tank3d(seed=3, nx=nx, ny=ny, nz=nz)
    s, *_ = _state(c, 7)
    s = 1.6 * s
    T = wec.Tank3(c, step=False)
    T.set(wec.F3_SIGMA, s)
    T.reinit(4, 0.11)
    ref = L3.Oracle3(c).reinit(s, 4, 0.11)
    assert rel(T.get(wec.F3_SIGMA), ref) < 1e-12
    T.close()


def test_chain_advect_reinit_materials():
    nx, ny, nz = 48, 16, 24
    c = synth.tank3d(seed=4, nx=nx, ny=ny, nz=nz)
    s, u, v, w = _state(c, 9)
    T = wec.Tank3(c, step=False)
    for fid, a in ((wec.F3_SIGMA, s), (wec.F3_U, u), (wec.F3_V, v), (wec.F3_W, w)):
        T.set(fid, a)
    O = L3.Oracle3(c)
    for step in range(3):
        t = step * 0.01
        T.advect(0.01, t)
        T.reinit(2, t + 0.01)
        s = O.reinit(O.advect(s, u, v, w, 0.01, t), 2, t + 0.01)
    zc = c["body"]["zc"]
    m, mo = T.materials(zc), O.materials(s, zc)
    assert rel(T.get(wec.F3_SIGMA), s) < 1e-11
    assert rel(m["rho"], mo["rho"]) < 1e-12
    T.close()


def test_full_size_tank_sampled_cells():
    # 512 x 256 x 256: the GPU advection and materials at every cell of the six
    # boundary layers' edges and corners plus 20000 random cells, against the
    # oracle evaluated at those cells only
    c = synth.tank3d(seed=0)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    s, u, v, w = _state(c, 11)
    T = wec.Tank3(c, step=False)
    for fid, a in ((wec.F3_SIGMA, s), (wec.F3_U, u), (wec.F3_V, v), (wec.F3_W, w)):
        T.set(fid, a)
    zc = c["body"]["zc"]
    m = T.materials(zc)
    T.advect(0.001, 0.5)
    out = T.get(wec.F3_SIGMA).ravel()
    rng = np.random.default_rng(0)
    idx = set(rng.integers(0, nx * ny * nz, 20000).tolist())
    for k in (0, 1, 2, nz - 3, nz - 2, nz - 1):
        for j in (0, 1, ny - 1):
            for i in (0, 1, 2, 3, nx - 3, nx - 1):
                idx.add((k * ny + j) * nx + i)
    cells = np.array(sorted(idx), dtype=np.int64)
    O = L3.Oracle3(c)
    ref = O.advect_cells(s, u, v, w, 0.001, 0.5, cells)
    assert np.max(np.abs(out[cells] - ref)) <= 1e-12 * np.max(np.abs(ref))
    # materials are pointwise: the oracle on a slab through the cylinder
    k0, k1 = int((zc - 0.6) / (c["lx"] / nx)), int((zc + 0.6) / (c["lx"] / nx))
    sub = dict(c, nz=k1 - k0, lz=(k1 - k0) * c["lx"] / nx)
    mo = L3.Oracle3(sub).materials(s[k0:k1], zc - k0 * c["lx"] / nx)
    for key in ("rho", "mu", "chi"):
        assert rel(m[key][k0:k1], mo[key]) < 1e-13, key
    assert np.count_nonzero(m["chi"] > 0.5) > 1000  # the cylinder is in the grid
    T.close()


def test_invalid_uses_are_errors():
    c = synth.tank3d(seed=0, nx=16, ny=8, nz=8)
    T = wec.Tank3(c, step=False)
    with pytest.raises(ValueError):
        T.set(wec.F3_SIGMA, np.zeros((8, 8, 15)))
    with pytest.raises(wec.WecError):  # materials are not settable
        wec._check(wec.load().wec_tank3_set_field(T.h, wec.F3_RHO, wec._ptr(np.zeros(8 * 8 * 16)), 8 * 8 * 16))
    with pytest.raises(wec.WecError):
        T.advect(-1.0, 0.0)
    T.close()
    bad = dict(c, lz=c["lz"] * 1.5)  # non-uniform grid
    with pytest.raises(wec.WecError):
        wec.Tank3(bad)
