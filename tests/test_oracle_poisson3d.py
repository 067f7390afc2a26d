"""Pins of the 3D pressure-Poisson oracle (the pressure equation of the
projection with d = 3, section "Continuous equations of motion"; solver and
multigrid as in two dimensions).  Each test states the fact it checks; none of
the expected values comes from the CUDA library.

- closed form: with unit coefficients the operator's eigenvectors are products
  of cosines (Neumann walls and bed, Dirichlet top), eigenvalues in closed form;
- reduction: a field constant along y (or along x) sees exactly the two-
  dimensional operator of the other two directions -- the 2D oracle, which has
  pins of its own -- and the 3D solution of such a problem is the 2D solution;
- brute force: the assembled matrix is symmetric positive definite with at most
  seven entries per row, and wall coefficients do not enter it; FGMRES reaches
  the dense direct solution of that matrix;
- second order on a manufactured variable-coefficient solution;
- the V-cycle contracts the error (spectral radius of I - M A well below 1,
  which the coarse-coefficient rule decides).
"""
import math

import numpy as np
import pytest

from oracle import poisson3d as O3
from oracle import tank as O2
from paper_2206_07732_gb300 import synth


def _unit(nx, ny, nz):
    bx, by, bz = np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)), np.ones((nz + 1, ny, nx))
    bx[:, :, 0] = bx[:, :, nx] = 0.0
    by[:, 0, :] = by[:, ny, :] = 0.0
    bz[0] = 0.0
    return bx, by, bz


def _assemble(bx, by, bz, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(shape)
    for q in range(n):
        e.flat[:] = 0.0
        e.flat[q] = 1.0
        A[:, q] = O3.apply(bx, by, bz, e).ravel()
    return A


@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 0, 2), (3, 2, 1), (7, 5, 6)])
def test_unit_coefficient_eigenpairs(mode):
    # v = cos(pi mx (i+1/2)/nx) cos(pi my (j+1/2)/ny) cos(pi (q+1/2)(k+1/2)/nz):
    # the Neumann ghost equals the cell value, the Dirichlet ghost its negative,
    # so A v = (4 sin^2(pi mx / 2nx) + 4 sin^2(pi my / 2ny) + 4 sin^2(pi (q+1/2) / 2nz)) v
    nx, ny, nz = 12, 10, 8
    mx, my, q = mode
    i, j, k = np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5
    v = (np.cos(math.pi * (q + 0.5) * k / nz)[:, None, None] * np.cos(math.pi * my * j / ny)[None, :, None] *
         np.cos(math.pi * mx * i / nx)[None, None, :])
    lam = sum(4.0 * math.sin(0.5 * math.pi * a) ** 2 for a in (mx / nx, my / ny, (q + 0.5) / nz))
    y = O3.apply(*_unit(nx, ny, nz), v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13 * max(lam, 1.0)


def test_levels_of_the_hierarchy():
    # halve every size while all three are even and at least 4
    assert O3.levels(512, 256, 256) == (8, (4, 2, 2))
    assert O3.levels(48, 24, 32) == (4, (6, 3, 4))
    assert O3.levels(40, 24, 16) == (4, (5, 3, 2))
    assert O3.levels(6, 4, 4) == (2, (3, 2, 2))


def test_y_invariant_field_is_the_2d_operator():
    # p(i, k) constant along y: the y faces see no difference, so A3 p = A2 p with
    # the 2D grid (x, vertical) = (x, z) and beta_u = beta_x, beta_v = beta_z
    nx, ny, nz = 10, 6, 8
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=4, contrast=50.0)
    bu2, bv2 = synth.random_coefficients(nx, nz, seed=5, contrast=50.0)
    bx[:] = bu2[:, None, :]
    bz[:] = bv2[:, None, :]
    p2 = np.random.default_rng(1).standard_normal((nz, nx))
    y3 = O3.apply(bx, by, bz, np.repeat(p2[:, None, :], ny, axis=1))
    y2 = O2.poisson_apply(bu2, bv2, p2)
    assert np.max(np.abs(y3 - y2[:, None, :])) <= 1e-14 * np.max(np.abs(y2))


def test_x_invariant_field_is_the_2d_operator():
    # p(j, k) constant along x: the 2D grid (x, vertical) = (y, z) with
    # beta_u = beta_y, beta_v = beta_z
    nx, ny, nz = 6, 12, 8
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=6, contrast=50.0)
    bu2, bv2 = synth.random_coefficients(ny, nz, seed=7, contrast=50.0)
    by[:] = bu2[:, :, None]
    bz[:] = bv2[:, :, None]
    p2 = np.random.default_rng(2).standard_normal((nz, ny))
    y3 = O3.apply(bx, by, bz, np.repeat(p2[:, :, None], nx, axis=2))
    y2 = O2.poisson_apply(bu2, bv2, p2)
    assert np.max(np.abs(y3 - y2[:, :, None])) <= 1e-14 * np.max(np.abs(y2))


def test_y_invariant_solve_is_the_2d_solve():
    nx, ny, nz = 32, 8, 16
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=8, contrast=1e3)
    bu2, bv2 = synth.random_coefficients(nx, nz, seed=9, contrast=1e3)
    bx[:] = bu2[:, None, :]
    bz[:] = bv2[:, None, :]
    b2 = np.random.default_rng(3).standard_normal((nz, nx))
    x3, info = O3.solve(bx, by, bz, np.repeat(b2[:, None, :], ny, axis=1), rtol=1e-12)
    x2, info2 = O2.poisson_solve(bu2, bv2, b2, rtol=1e-12)
    assert info["status"] == 0 and info2["status"] == 0
    assert np.max(np.abs(x3 - x2[:, None, :])) <= 1e-8 * np.max(np.abs(x2))


def test_matrix_is_spd_seven_point_and_ignores_walls():
    nx, ny, nz = 4, 4, 6
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=10, contrast=1e2)
    A = _assemble(bx, by, bz, (nz, ny, nx))
    assert np.array_equal(A, A.T)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    assert max(np.count_nonzero(A[r]) for r in range(A.shape[0])) <= 7
    # off-diagonal entries are minus the shared face's coefficient
    c = lambda i, j, k: (k * ny + j) * nx + i
    assert A[c(1, 2, 3), c(2, 2, 3)] == -bx[3, 2, 2]
    assert A[c(1, 2, 3), c(1, 3, 3)] == -by[3, 3, 1]
    assert A[c(1, 2, 3), c(1, 2, 4)] == -bz[4, 2, 1]
    # the top layer's diagonal counts its top face twice
    assert A[c(2, 1, nz - 1), c(2, 1, nz - 1)] == pytest.approx(
        bx[nz - 1, 1, 2] + bx[nz - 1, 1, 3] + by[nz - 1, 1, 2] + by[nz - 1, 2, 2] + bz[nz - 1, 1, 2] +
        2 * bz[nz, 1, 2], rel=1e-15)
    wx, wy, wz = bx.copy(), by.copy(), bz.copy()
    wx[:, :, 0] = wx[:, :, nx] = 9.0
    wy[:, 0, :] = wy[:, ny, :] = 9.0
    wz[0] = 9.0
    assert np.array_equal(_assemble(wx, wy, wz, (nz, ny, nx)), A)


@pytest.mark.parametrize("contrast", [1.0, 1e4])
def test_solver_matches_dense(contrast):
    nx, ny, nz = 8, 4, 8
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=11, contrast=contrast)
    A = _assemble(bx, by, bz, (nz, ny, nx))
    b = np.random.default_rng(4).standard_normal((nz, ny, nx))
    x_ref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    x, info = O3.solve(bx, by, bz, b, rtol=1e-13)
    assert info["status"] == 0 and info["relres"] <= 1e-13
    assert np.max(np.abs(x - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))


def test_manufactured_second_order():
    # -div(beta grad p) = f, p = cos(pi x / Lx) cos(pi y / Ly) cos(pi z / (2 Lz)):
    # Neumann on the walls and the bed, p = 0 on the top; discrete error ~ h^2
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z")
    Lx, Ly, Lz = 2.0, 1.0, 1.0
    p = sp.cos(sp.pi * X / Lx) * sp.cos(sp.pi * Y / Ly) * sp.cos(sp.pi * Z / (2 * Lz))
    beta = 1 + sp.Rational(1, 2) * sp.sin(X) * sp.sin(2 * Y) ** 2 * sp.cos(Z)
    f = -sum(sp.diff(beta * sp.diff(p, s), s) for s in (X, Y, Z))
    pf, bf, ff = (sp.lambdify((X, Y, Z), e, "numpy") for e in (p, beta, f))
    errs = []
    for nx in (16, 32, 64):
        ny, nz = nx // 2, nx // 2
        h = Lx / nx
        c = lambda m: (np.arange(m) + 0.5) * h
        fc = lambda m: np.arange(m + 1) * h
        mesh = lambda zs, ys, xs: np.meshgrid(zs, ys, xs, indexing="ij")
        Zx, Yx, Xx = mesh(c(nz), c(ny), fc(nx))
        Zy, Yy, Xy = mesh(c(nz), fc(ny), c(nx))
        Zz, Yz, Xz = mesh(fc(nz), c(ny), c(nx))
        Zc, Yc, Xc = mesh(c(nz), c(ny), c(nx))
        bx, by, bz = bf(Xx, Yx, Zx), bf(Xy, Yy, Zy), bf(Xz, Yz, Zz)
        bx[:, :, 0] = bx[:, :, nx] = 0.0
        by[:, 0, :] = by[:, ny, :] = 0.0
        bz[0] = 0.0
        x, info = O3.solve(bx, by, bz, h * h * ff(Xc, Yc, Zc), rtol=1e-11)
        assert info["status"] == 0
        errs.append(np.max(np.abs(x - pf(Xc, Yc, Zc))))
    rates = [math.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert min(rates) > 1.8, (errs, rates)


@pytest.mark.parametrize("contrast", [1.0, 10.0])
def test_vcycle_contracts(contrast):
    # one V(2,2)-cycle as a stationary iteration x += M (b - A x): spectral radius
    # of I - M A.  With the half-sum coarse coefficients it is 0.10 (contrast 1)
    # and 0.19 (contrast 10); a coarse operator off by a factor of two gives 2.4 /
    # 2.1 (mean of the four faces: divergent) or 0.66 / 0.70 (their plain sum),
    # measured on the same cases.
    nx, ny, nz = 16, 8, 8
    bx, by, bz = synth.random_coefficients3(nx, ny, nz, seed=12, contrast=contrast)
    A = _assemble(bx, by, bz, (nz, ny, nx))
    n = A.shape[0]
    M = np.zeros_like(A)
    e = np.zeros((nz, ny, nx))
    for q in range(n):
        e.flat[:] = 0.0
        e.flat[q] = 1.0
        M[:, q] = O3.vcycle(bx, by, bz, e)[0].ravel()
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(n) - M @ A)))
    print(f"contrast {contrast}: spectral radius {rho:.3f}")
    assert rho < 0.3
