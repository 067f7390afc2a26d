"""Pins of the oracle's discretisation against closed forms, invariants, brute force.

Each test states the paper passage (or the mathematical fact) it pins.  None of the
expected values comes from the CUDA library.
"""
import math

import numpy as np
import pytest

from oracle import tank as O
from paper_2206_07732_gb300 import synth


def _tank(nx=64, ny=32, body=False, H=0.0, **kw):
    c = synth.still_water(nx=nx, ny=ny, body=body, **kw)
    c["wave"]["H"] = H
    return c


# ------------------------------------------------------------ materials -----
def test_heaviside_points():
    # Eqs. Hflow / Hbody: 0 below -eps, 1 above eps, 1/2 at 0, C1 at +-eps
    eps = 0.1
    assert O.heaviside(-eps * 1.0000001, eps) == 0.0
    assert O.heaviside(eps * 1.0000001, eps) == 1.0
    assert O.heaviside(0.0, eps) == 0.5
    assert O.heaviside(-eps, eps) == pytest.approx(0.0, abs=1e-16)
    assert O.heaviside(eps, eps) == pytest.approx(1.0, abs=1e-16)
    xs = np.linspace(-eps, eps, 101)
    hs = np.array([O.heaviside(x, eps) for x in xs])
    assert np.all(np.diff(hs) >= 0)
    d = 1e-7
    slope = (O.heaviside(eps, eps) - O.heaviside(eps - d, eps)) / d
    assert abs(slope) < 1e-4  # zero slope where it meets the constant branch
    # symmetric about 0: H(x) + H(-x) = 1
    for x in (0.013, 0.05, 0.09):
        assert O.heaviside(x, eps) + O.heaviside(-x, eps) == pytest.approx(1.0, abs=1e-15)


def test_materials_two_stage():
    # Eqs. ls_flow, ls_solid: water below the surface, air above, solid in the body
    cfg = _tank(body=True)
    T = O.OracleTank(cfg)
    m = T.materials()
    h = cfg["lx"] / cfg["nx"]
    b = cfg["body"]
    rho_s = b["mass"] / (b["width"] * b["height"])
    y = (np.arange(cfg["ny"]) + 0.5) * h
    x = (np.arange(cfg["nx"]) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    psi = np.maximum(np.abs(X - b["xc"]) - 0.5 * b["width"], np.abs(Y - b["yc"]) - 0.5 * b["height"])
    sig = Y - cfg["depth"]
    water = (sig < -h) & (psi > h)
    air = (sig > h) & (psi > h)
    solid = psi < -h
    assert water.any() and air.any() and solid.any()
    # (rho_s + (rho_f - rho_s) 1 rounds to rho_f within a few ulps)
    np.testing.assert_allclose(m["rho"][water], cfg["rho_w"], rtol=1e-13)
    np.testing.assert_allclose(m["rho"][air], cfg["rho_a"], rtol=1e-13)
    np.testing.assert_allclose(m["rho"][solid], rho_s, rtol=1e-15)
    np.testing.assert_allclose(m["mu"][water], cfg["mu_w"], rtol=1e-13)
    np.testing.assert_allclose(m["mu"][air], cfg["mu_a"], rtol=1e-13)
    assert np.all(m["chi"][solid] == 1.0) and np.all(m["chi"][water | air] == 0.0)
    # flow density ignores the body (gravity term uses rho^flow)
    assert np.all(m["rho_flow"][solid & (sig < -h)] == cfg["rho_w"])


# ---------------------------------------------------------------- inflow -----
def test_inflow_is_linear_potential_flow():
    # Section "Numerical wave tank": Dirichlet Airy velocities.  For a tiny
    # amplitude (stretching ~ identity) the field is divergence free, irrotational,
    # has v = 0 on the bed and meets the linear kinematic surface condition.
    cfg = synth.tank_small(seed=3)
    cfg["wave"]["H"] = 2e-7
    T = O.OracleTank(cfg)
    d, e, t = cfg["depth"], 1e-5, 0.37
    for (x, y) in [(0.3, 0.2), (1.1, 0.6), (2.0, 0.85)]:
        u_xp, _ = T.inflow(x + e, y, t); u_xm, _ = T.inflow(x - e, y, t)
        _, v_yp = T.inflow(x, y + e, t); _, v_ym = T.inflow(x, y - e, t)
        u_yp, _ = T.inflow(x, y + e, t); u_ym, _ = T.inflow(x, y - e, t)
        _, v_xp = T.inflow(x + e, y, t); _, v_xm = T.inflow(x - e, y, t)
        scale = abs(T.inflow(x, y, t)[0]) + abs(T.inflow(x, y, t)[1]) + 1e-30
        div = (u_xp - u_xm + v_yp - v_ym) / (2 * e)
        rot = (u_yp - u_ym - v_xp + v_xm) / (2 * e)
        assert abs(div) < 1e-5 * scale / e * e * 10 + 1e-9 * scale / e
        assert abs(rot) < 1e-5 * scale / e * e * 10 + 1e-9 * scale / e
    assert T.inflow(0.0, 0.0, t)[1] == 0.0
    # kinematic condition v = d eta / dt at the still-water level (linear)
    a, w, k, ph = 0.5 * cfg["wave"]["H"], 2 * math.pi / cfg["wave"]["T"], None, cfg["wave"]["phase"]
    from oracle import waves as W
    k = W.dispersion_k(w, d, cfg["g"])
    x = 0.7
    deta_dt = a * w * math.sin(k * x - w * t + ph)
    # (at the surface the air blend 1 - H(0) = 1/2 halves it)
    assert T.inflow(x, d - 1e-12, t)[1] == pytest.approx(0.5 * deta_dt, rel=1e-5)
    # zero above the smoothed surface
    assert T.inflow(x, d + 0.2, t) == (0.0, 0.0)


# -------------------------------------------------------------- advection -----
def _set_uniform_velocity(T, uc, vc):
    u = np.full(T.shape(O.F_U), uc)
    v = np.full(T.shape(O.F_V), vc)
    T.set(O.F_U, u)
    T.set(O.F_V, v)


def test_advect_linear_field_exact():
    # PPM reproduces a linear field exactly: sigma - dt (u a + v b)
    cfg = _tank(nx=48, ny=32)
    T = O.OracleTank(cfg)
    h = cfg["lx"] / cfg["nx"]
    x = (np.arange(cfg["nx"]) + 0.5) * h
    y = (np.arange(cfg["ny"]) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    a, b, c = 0.3, -0.7, 0.25
    T.set(O.F_SIGMA, a * X + b * Y + c)
    _set_uniform_velocity(T, 0.8, -0.45)
    dt = 0.01
    T.advect(dt)
    got = T.get(O.F_SIGMA)
    want = a * X + b * Y + c - dt * (0.8 * a - 0.45 * b)
    # left three columns see the wave ghost, right three the zero-gradient wall
    np.testing.assert_allclose(got[:, 3:-3], want[:, 3:-3], rtol=0, atol=1e-13)


def test_advect_translation_order():
    # smooth bump translated by a uniform velocity: error falls ~h^2 or faster
    errs = []
    for nx in (64, 128):
        ny = nx // 2
        cfg = _tank(nx=nx, ny=ny)
        T = O.OracleTank(cfg)
        h = cfg["lx"] / nx
        x = (np.arange(nx) + 0.5) * h
        y = (np.arange(ny) + 0.5) * h
        X, Y = np.meshgrid(x, y)
        f = lambda X, Y: np.exp(-((X - 1.6) ** 2 + (Y - 1.0) ** 2) / 0.4 ** 2)
        T.set(O.F_SIGMA, f(X, Y))
        uc, vc = 0.6, 0.3
        _set_uniform_velocity(T, uc, vc)
        # small CFL (0.02, the tank runs near 0.01): the single-stage unsplit update
        # has an O(dt) cross-term error, so spatial order shows only when dt << h
        tend, nsteps = 0.5, int(round(0.5 / (0.02 * h / 0.6)))
        dt = tend / nsteps
        for _ in range(nsteps):
            T.advect(dt)
        err = T.get(O.F_SIGMA) - f(X - uc * tend, Y - vc * tend)
        mask = (np.abs(X - 1.9) < 0.5) & (np.abs(Y - 1.15) < 0.5)
        errs.append((np.max(np.abs(err[mask])), np.mean(np.abs(err[mask]))))
    # the limiter clips the bump's peak (standard PPM is not extremum preserving),
    # so the max norm converges a little slower than the mean error
    assert errs[1][0] < errs[0][0] / 3.0, errs
    assert errs[1][1] < errs[0][1] / 3.5, errs


def test_advect_constant_preserved():
    cfg = _tank(nx=48, ny=32)
    T = O.OracleTank(cfg)
    T.set(O.F_SIGMA, np.full(T.shape(O.F_SIGMA), 0.37))
    rng = np.random.default_rng(5)
    T.set(O.F_U, rng.standard_normal(T.shape(O.F_U)))
    T.set(O.F_V, rng.standard_normal(T.shape(O.F_V)))
    T.advect(1e-3)
    got = T.get(O.F_SIGMA)
    assert np.all(got[:, 3:] == 0.37)


# ---------------------------------------------------------- reinitialisation -----
def test_reinit_flat_interface_fixed_point():
    # sigma = y - d is already a signed distance: |grad| = 1, so it must not move
    cfg = _tank(nx=48, ny=32)
    T = O.OracleTank(cfg)
    s0 = T.get(O.F_SIGMA)
    T.reinit(20)
    np.testing.assert_allclose(T.get(O.F_SIGMA), s0, rtol=0, atol=1e-14)


def test_reinit_restores_unit_gradient():
    # Sussman relaxation: a distorted distance function relaxes toward |grad| = 1
    # near the interface while the zero contour stays put.
    nx, ny = 96, 48
    cfg = _tank(nx=nx, ny=ny)
    T = O.OracleTank(cfg)
    h = cfg["lx"] / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    R, x0, y0 = 0.5, 2.0, 0.9
    r = np.hypot(X - x0, Y - y0)
    s = (r - R) * (1.0 + 0.5 * (X - x0)) * 2.0  # wrong slope, still zero on the circle
    T.set(O.F_SIGMA, s)
    T.reinit(60)
    g = T.get(O.F_SIGMA)
    gy, gx = np.gradient(g, h)
    band = (np.abs(r - R) < 3 * h) & (np.abs(X - x0) < 1.0)
    gn = np.hypot(gx, gy)[band]
    assert np.mean(np.abs(gn - 1.0)) < 0.05
    # zero contour: sigma at the exact circle points, interpolated bilinearly
    from scipy.interpolate import RegularGridInterpolator
    ip = RegularGridInterpolator((y, x), g)
    th = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    pts = np.stack([y0 + R * np.sin(th), x0 + R * np.cos(th)], axis=1)
    assert np.max(np.abs(ip(pts))) < 0.25 * h


# --------------------------------------------------------------- Poisson -----
def _assemble(bu, bv, nx, ny):
    n = nx * ny
    A = np.zeros((n, n))
    e = np.zeros((ny, nx))
    for k in range(n):
        e.flat[:] = 0.0
        e.flat[k] = 1.0
        A[:, k] = O.poisson_apply(bu, bv, e).ravel()
    return A


@pytest.mark.parametrize("contrast", [1.0, 1e5])
def test_poisson_solver_matches_dense(contrast):
    # FGMRES + V-cycle reaches the dense direct solution of the same operator
    nx, ny = 16, 8
    bu, bv = synth.random_coefficients(nx, ny, seed=7, contrast=contrast)
    A = _assemble(bu, bv, nx, ny)
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.all(np.linalg.eigvalsh(A) > 0)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((ny, nx))
    x_ref = np.linalg.solve(A, b.ravel()).reshape(ny, nx)
    x, info = O.poisson_solve(bu, bv, b, rtol=1e-13)
    assert info["status"] == 0
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))


def test_poisson_operator_stencil_brute_force():
    # each row of A: diag = sum of the cell's face coefficients (Neumann walls
    # drop out, the top face counts twice), off-diagonals = -beta of the shared face
    nx, ny = 5, 4
    bu, bv = synth.random_coefficients(nx, ny, seed=11)
    bu[:, 0] = 9.0  # wall coefficients are ignored whatever they hold
    bu[:, nx] = 9.0
    bv[0, :] = 9.0
    A = _assemble(bu, bv, nx, ny)
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            d = (bu[j, i] if i > 0 else 0) + (bu[j, i + 1] if i < nx - 1 else 0) + \
                (bv[j, i] if j > 0 else 0) + (bv[j + 1, i] if j < ny - 1 else 2 * bv[j + 1, i])
            assert A[r, r] == pytest.approx(d, rel=1e-15)
            if i > 0:
                assert A[r, r - 1] == -bu[j, i]
            if j < ny - 1:
                assert A[r, r + nx] == -bv[j + 1, i]
            assert np.count_nonzero(A[r]) <= 5


def test_poisson_manufactured_second_order():
    # -div(beta grad p) = f with p = cos(pi x / Lx) cos(pi y / (2 Ly)): Neumann on
    # the left/right/bottom walls, p = 0 on the top.  Discrete error ~ h^2.
    sp = pytest.importorskip("sympy")
    xs, ys = sp.symbols("x y")
    Lx, Ly = 2.0, 1.0
    p = sp.cos(sp.pi * xs / Lx) * sp.cos(sp.pi * ys / (2 * Ly))
    beta = 1 + sp.Rational(1, 2) * sp.sin(xs) * sp.sin(2 * ys) ** 2
    f = -(sp.diff(beta * sp.diff(p, xs), xs) + sp.diff(beta * sp.diff(p, ys), ys))
    pf, bf, ff = (sp.lambdify((xs, ys), e, "numpy") for e in (p, beta, f))
    errs = []
    for nx in (16, 32, 64, 128):
        ny = nx // 2
        h = Lx / nx
        xc = (np.arange(nx) + 0.5) * h
        yc = (np.arange(ny) + 0.5) * h
        Xc, Yc = np.meshgrid(xc, yc)
        Xu, Yu = np.meshgrid(np.arange(nx + 1) * h, yc)
        Xv, Yv = np.meshgrid(xc, np.arange(ny + 1) * h)
        bu = bf(Xu, Yu) * np.ones_like(Xu)
        bv = bf(Xv, Yv) * np.ones_like(Xv)
        bu[:, 0] = bu[:, nx] = 0.0
        bv[0, :] = 0.0
        b = h * h * ff(Xc, Yc)
        x, info = O.poisson_solve(bu, bv, b, rtol=1e-12)
        assert info["status"] == 0
        errs.append(np.max(np.abs(x - pf(Xc, Yc))))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert min(rates) > 1.8, (errs, rates)


def test_vcycle_contracts():
    # one V-cycle as a stationary iteration: error contraction < 1 (spectral radius)
    nx, ny = 32, 16
    bu, bv = synth.random_coefficients(nx, ny, seed=3)
    A = _assemble(bu, bv, nx, ny)
    M = np.zeros_like(A)
    e = np.zeros((ny, nx))
    for k in range(nx * ny):
        e.flat[:] = 0.0
        e.flat[k] = 1.0
        M[:, k] = O.vcycle(bu, bv, e)[0].ravel()
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(nx * ny) - M @ A)))
    assert rho < 0.5


# ------------------------------------------------------------- transport -----
def _faces(cfg):
    h = cfg["lx"] / cfg["nx"]
    nx, ny = cfg["nx"], cfg["ny"]
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    Xu, Yu = np.meshgrid(np.arange(nx + 1) * h, yc)
    Xv, Yv = np.meshgrid(xc, np.arange(ny + 1) * h)
    Xc, Yc = np.meshgrid(xc, yc)
    return h, (Xc, Yc), (Xu, Yu), (Xv, Yv)


def test_transport_linear_fields_exact():
    # consistent transport (Eq. c_discrete_momentum): for a linear divergence-free
    # velocity and a linear density, rho-breve = rho - dt u.grad(rho) and
    # C = div(rho u (x) u) hold exactly at interior faces.
    cfg = _tank(nx=32, ny=24)
    T = O.OracleTank(cfg)
    h, (Xc, Yc), (Xu, Yu), (Xv, Yv) = _faces(cfg)
    a, u0, v0 = 0.4, 0.3, -0.2
    T.set(O.F_U, u0 + a * Xu)
    T.set(O.F_V, v0 - a * Yv)
    r0, rx, ry = 2.0, 0.3, -0.5
    rho = r0 + rx * Xc + ry * Yc
    dt = 1e-3
    rbu, rbv, Cu, Cv = T.transport(rho, dt)
    sl = (slice(3, -3), slice(3, -3))
    Uf = lambda X, Y: u0 + a * X
    Vf = lambda X, Y: v0 - a * Y
    Rf = lambda X, Y: r0 + rx * X + ry * Y
    for (X, Y, rb, Cc, comp) in [(Xu, Yu, rbu, Cu, 0), (Xv, Yv, rbv, Cv, 1)]:
        # mass flux rho u is quadratic: its face difference is the exact divergence
        want_rb = Rf(X, Y) - dt * (Uf(X, Y) * rx + Vf(X, Y) * ry)
        np.testing.assert_allclose(rb[sl], want_rb[sl], rtol=0, atol=1e-13)
        # the limited reconstructions are exact for linear fields, so C is the exact
        # finite-volume difference of the analytic flux rho u q over the CV
        q = Uf if comp == 0 else Vf
        Fx = lambda X, Y: Rf(X, Y) * Uf(X, Y) * q(X, Y)
        Fy = lambda X, Y: Rf(X, Y) * Vf(X, Y) * q(X, Y)
        want_C = (Fx(X + h / 2, Y) - Fx(X - h / 2, Y)) / h + (Fy(X, Y + h / 2) - Fy(X, Y - h / 2)) / h
        np.testing.assert_allclose(Cc[sl], want_C[sl], rtol=0, atol=1e-12)
        # ... which differs from rho (u.grad) q + q u.grad rho only by h^2/24 f'''
        cont = Rf(X, Y) * (Uf(X, Y) * (a if comp == 0 else 0.0) + Vf(X, Y) * (0.0 if comp == 0 else -a)) \
            + q(X, Y) * (Uf(X, Y) * rx + Vf(X, Y) * ry)
        assert np.max(np.abs(Cc[sl] - cont[sl])) < h * h


def test_transport_uniform_density_stays():
    cfg = _tank(nx=32, ny=24)
    T = O.OracleTank(cfg)
    rng = np.random.default_rng(9)
    T.set(O.F_U, rng.standard_normal(T.shape(O.F_U)))
    T.set(O.F_V, rng.standard_normal(T.shape(O.F_V)))
    # a uniform density is carried unchanged only by a divergence-free field;
    # with a zero field it stays exactly and C vanishes
    T.set(O.F_U, np.zeros(T.shape(O.F_U)))
    T.set(O.F_V, np.zeros(T.shape(O.F_V)))
    rbu, rbv, Cu, Cv = T.transport(np.full((24, 32), 7.0), 1e-3)
    assert np.all(rbu[:, 1:-1] == 7.0) and np.all(rbv[1:, :] == 7.0)
    assert np.all(Cu == 0.0) and np.all(Cv == 0.0)


# --------------------------------------------------------------- viscous -----
@pytest.mark.parametrize("case", ["u_xx", "u_yy", "v_xx", "v_yy", "xy"])
def test_viscous_polynomials(case):
    # L_mu u = div[mu (grad u + grad u^T)] = mu (lap u + grad div u) for uniform mu
    cfg = _tank(nx=24, ny=16)
    T = O.OracleTank(cfg)
    h, (Xc, Yc), (Xu, Yu), (Xv, Yv) = _faces(cfg)
    mu = 0.7
    U = {"u_xx": Xu ** 2, "u_yy": Yu ** 2, "v_xx": 0 * Xu, "v_yy": 0 * Xu, "xy": Xu * Yu}[case]
    V = {"u_xx": 0 * Xv, "u_yy": 0 * Xv, "v_xx": Xv ** 2, "v_yy": Yv ** 2, "xy": 0 * Xv}[case]
    want = {"u_xx": (4 * mu, 0.0), "u_yy": (2 * mu, 0.0), "v_xx": (0.0, 2 * mu),
            "v_yy": (0.0, 4 * mu), "xy": (0.0, mu)}[case]
    T.set(O.F_U, U)
    T.set(O.F_V, V)
    Lx, Ly = T.viscous(np.full((16, 24), mu))
    np.testing.assert_allclose(Lx[2:-2, 2:-2], want[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(Ly[2:-2, 2:-2], want[1], rtol=0, atol=1e-9)


# ----------------------------------------------------------------- force -----
def _stair_extent(cfg):
    h = cfg["lx"] / cfg["nx"]
    b = cfg["body"]
    xc = (np.arange(cfg["nx"]) + 0.5) * h
    yc = (np.arange(cfg["ny"]) + 0.5) * h
    cols = np.abs(xc - b["xc"]) - 0.5 * b["width"] < 0
    rows = np.abs(yc - b["yc"]) - 0.5 * b["height"] < 0
    return cols.sum() * h, rows, h


def test_force_linear_pressure_exact():
    # Eq. int_fh with p = P0 - rho g y: the |psi|-weighted face pressure is the
    # exact pressure at the body surface, so F = rho g W B (W: stair-step width)
    # In a corner column the CSG max is set by the side distance, which is not
    # linear along y; the body is placed so that no bottom/top cell is closer to
    # a side than to the bottom/top (h = 1/16, box edges at y = 0.83, 1.23).
    cfg = _tank(nx=64, ny=32, body=True)
    cfg["body"]["yc"] = 1.03
    T = O.OracleTank(cfg)
    h, (Xc, Yc), _, _ = _faces(cfg)
    rho, g = 1000.0, 9.81
    T.set(O.F_P, 5000.0 - rho * g * Yc)
    T.set(O.F_U, np.zeros(T.shape(O.F_U)))
    T.set(O.F_V, np.zeros(T.shape(O.F_V)))
    W_, _, _ = _stair_extent(cfg)
    F = T.force()
    assert F == pytest.approx(rho * g * W_ * cfg["body"]["height"], rel=1e-12)


def test_force_viscous_quadratic_exact():
    # Eq. int_fh viscous part: v = c y^2, u = 0, uniform mu, p = 0.  Only the
    # y-faces contribute 2 mu dv/dy n_y: F = 4 mu c W (y_top - y_bottom) of the
    # stair-step faces.
    cfg = _tank(nx=64, ny=32, body=True)
    cfg["mu_a"] = cfg["mu_w"]
    T = O.OracleTank(cfg)
    h, (Xc, Yc), _, (Xv, Yv) = _faces(cfg)
    T.set(O.F_SIGMA, -np.ones(T.shape(O.F_SIGMA)))  # all water: uniform mu
    T.set(O.F_P, np.zeros(T.shape(O.F_P)))
    T.set(O.F_U, np.zeros(T.shape(O.F_U)))
    c = 0.3
    T.set(O.F_V, c * Yv ** 2)
    W_, rows, h = _stair_extent(cfg)
    jb = np.argmax(rows)
    jt = len(rows) - np.argmax(rows[::-1])
    F = T.force()
    assert F == pytest.approx(4 * cfg["mu_w"] * c * W_ * (jt - jb) * h, rel=1e-10)


# ------------------------------------------------------- step invariants -----
def test_still_water_stays_at_rest():
    # hydrostatic balance is exact on the MAC grid: gravity uses the flow density,
    # p starts from its discrete hydrostatic profile
    cfg = _tank(nx=64, ny=32, rtol=1e-12)
    T = O.OracleTank(cfg)
    for _ in range(30):
        r = T.step(cfg["dt"])
        assert r["status"] == 0
    assert np.max(np.abs(T.get(O.F_U))) < 1e-10
    assert np.max(np.abs(T.get(O.F_V))) < 1e-10


def test_divergence_below_solver_tolerance():
    # Eq. c_discrete_continuity: h div u^{n+1} = A p - b, so ||h div u|| <= rtol ||b||
    cfg = synth.tank_small(seed=1, nx=64, ny=32)
    T = O.OracleTank(cfg)
    for _ in range(5):
        r = T.step(cfg["dt"])
    u, v, b = T.get(O.F_U), T.get(O.F_V), T.get(O.F_RHS)
    h = cfg["lx"] / cfg["nx"]
    div = h * (u[:, 1:] - u[:, :-1] + v[1:, :] - v[:-1, :])
    assert np.linalg.norm(div) <= 1.01 * cfg["solver"]["rtol"] * np.linalg.norm(b)
    assert np.linalg.norm(div) == pytest.approx(r["div_norm"], rel=1e-6)


def test_brinkman_enforces_rigid_velocity():
    # Eq. bp_discrete: inside the body u -> u_b = (0, zdot) as kappa_p -> 0
    cfg = synth.tank_small(seed=2, nx=64, ny=32)
    T = O.OracleTank(cfg)
    for _ in range(10):
        T.step(cfg["dt"])
    m = T.materials()
    zd = T.body()["zdot"]
    v = T.get(O.F_V)
    u = T.get(O.F_U)
    inside = m["chi"] == 1.0
    vin = 0.5 * (v[1:, :] + v[:-1, :])[inside]
    uin = 0.5 * (u[:, 1:] + u[:, :-1])[inside]
    scale = max(abs(zd), 1e-3)
    assert np.max(np.abs(vin - zd)) < 0.05 * scale
    assert np.max(np.abs(uin)) < 0.05 * scale


def test_floating_box_static_force_archimedes():
    # Section "Fluid-structure coupling": at its floating draft the box's force
    # balances its weight (exact hydrostatics through the face interpolation)
    cfg = _tank(nx=64, ny=32, body=True)
    T = O.OracleTank(cfg)
    r = T.step(cfg["dt"])
    m = cfg["body"]["mass"]
    assert r["f_hydro"] == pytest.approx(m * cfg["g"], rel=5e-3)
    for _ in range(20):
        r = T.step(cfg["dt"])
    assert r["f_hydro"] == pytest.approx(m * cfg["g"], rel=5e-3)
    assert abs(r["zdot"]) < 1e-3


@pytest.mark.slow
def test_released_box_settles_to_draft():
    # released 2 cm low with a damper, the box returns toward its Archimedes draft
    cfg = _tank(nx=64, ny=32, body=True)
    cfg["body"] = synth.box_body(2.0, 0.5, 0.4, 0.2, 1.0, cfg["rho_w"], pto_damping=400.0,
                                 extra_sink=0.02)
    T = O.OracleTank(cfg)
    zs = []
    for n in range(1500):
        r = T.step(2e-3)
        assert r["status"] == 0
        zs.append(r["z"])
    h = cfg["lx"] / cfg["nx"]
    # equilibrium is z = +0.02 (back at the draft); within a quarter cell
    assert abs(np.mean(zs[-100:]) - 0.02) < 0.25 * h
    assert zs[0] > 0.0


def test_step_is_deterministic():
    cfg = synth.tank_small(seed=4, nx=64, ny=32)
    T1, T2 = O.OracleTank(cfg), O.OracleTank(cfg)
    for _ in range(3):
        a, b = T1.step(cfg["dt"]), T2.step(cfg["dt"])
    assert a == b
    assert np.array_equal(T1.get(O.F_P), T2.get(O.F_P))
