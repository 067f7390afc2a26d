"""Seeded synthetic inputs for the wave-tank workloads.

This module only draws random numbers and holds the workload definitions
(grid sizes, fluid constants, wave and body parameters).  It contains none of
the method's arithmetic: wave spectra, dispersion, materials, the time step and
the pressure solve live in the CUDA library (and, independently, in the CPU
oracle used by the tests).  Both sides receive the dictionaries built here.

Fluid constants and tank geometry follow the paper's numerical wave tank
(Section "Numerical wave tank", water/air properties of the test cases); the
sizes are the workloads this library is benchmarked on.
"""
from __future__ import annotations

import math

import numpy as np

WATER = dict(rho_w=1025.0, mu_w=1.0e-3)
AIR = dict(rho_a=1.225, mu_a=1.8e-5)
GRAVITY = 9.81


def _base(nx, ny, lx, ly, depth):
    d = dict(nx=nx, ny=ny, lx=lx, ly=ly, depth=depth, g=GRAVITY)
    d.update(WATER)
    d.update(AIR)
    return d


def _solver(rtol=1e-8, precision=0):
    return dict(rtol=rtol, max_iters=400, restart=20, n_reinit=4, n_jacobi=3,
                mg_pre=2, mg_post=2, precision=precision)


def box_body(xc, width, height, draft, depth, rho_w, pto_damping=0.0,
             kappa_p=1e-8, extra_sink=0.0):
    """Heaving box whose mass floats it at ``draft`` (per unit span).

    The mass is the workload's definition of the body ("mass giving a draft"),
    i.e. the displaced water mass per unit span; ``extra_sink`` shifts the
    initial position downward from that equilibrium.
    """
    mass = rho_w * width * draft
    yc = depth - draft + 0.5 * height - extra_sink
    # Artificial added mass of the stabilised heave update: the water mass that
    # would fill the box's rectangle (an upper scale of the 2D heave added mass).
    added_mass = rho_w * width * height
    return dict(xc=xc, yc=yc, width=width, height=height, mass=mass,
                added_mass=added_mass, kappa_p=kappa_p, pto_damping=pto_damping)


def regular_wave(H, T, rng):
    """One Airy component: height H, period T, phase drawn from ``rng``."""
    return dict(kind="regular", H=H, T=T, phase=float(rng.uniform(0.0, 2.0 * math.pi)))


def irregular_wave(Hs, Tp, gamma, ncomp, rng):
    """JONSWAP sea state; only the random phases are drawn here."""
    return dict(kind="jonswap", Hs=Hs, Tp=Tp, gamma=gamma, ncomp=ncomp,
                phases=rng.uniform(0.0, 2.0 * math.pi, size=ncomp).tolist())


def tank_small(seed=0, nx=128, ny=64, **solver_kw):
    """4 m x 2 m tank, 128x64, depth 1 m, regular wave H=0.05 T=1.0, box at x=2 m."""
    rng = np.random.default_rng(seed)
    c = _base(nx, ny, 4.0, 2.0, 1.0)
    c["wave"] = regular_wave(0.05, 1.0, rng)
    c["damp_x0"], c["damp_len"], c["probe_x"] = 3.0, 1.0, 0.5
    c["body"] = box_body(2.0, 0.5, 0.4, 0.2, 1.0, c["rho_w"], pto_damping=50.0)
    c["solver"] = _solver(**solver_kw)
    c["dt"], c["steps"] = 1e-3, 100
    c["name"] = f"tank {nx}x{ny} 4mx2m regular-wave box"
    return c


def tank_large(seed=0, nx=1024, ny=256, **solver_kw):
    """16 m x 4 m tank, 1024x256, depth 2.5 m, JONSWAP Hs=0.15 Tp=1.6 gamma=3.3, 64 comps."""
    rng = np.random.default_rng(seed)
    c = _base(nx, ny, 16.0, 4.0, 2.5)
    c["wave"] = irregular_wave(0.15, 1.6, 3.3, 64, rng)
    # Damping zone: 1.5 peak wavelengths (deep-water estimate g Tp^2 / 2pi).
    lam_p = GRAVITY * 1.6 ** 2 / (2.0 * math.pi)
    c["damp_len"] = 1.5 * lam_p
    c["damp_x0"] = 16.0 - c["damp_len"]
    c["probe_x"] = 1.0
    # Device placed one wavelength plus five half-widths from the inlet.
    c["body"] = box_body(lam_p + 2.5, 1.0, 0.8, 0.4, 2.5, c["rho_w"], pto_damping=0.0)
    c["solver"] = _solver(**solver_kw)
    c["dt"], c["steps"] = 5e-4, 2000
    c["pto_limit"] = 2000.0
    c["name"] = f"tank {nx}x{ny} 16mx4m JONSWAP box"
    return c


def tank_learned(seed=0, nx=512, ny=256, **solver_kw):
    """Training tanks of the learned warm start: the 1024x256 JONSWAP physics
    (h = 1/64 m, depth 2.5 m, box 1 m x 0.8 m at half draft) on an 8 m x 4 m
    tank, 512x256, with the sea state drawn from the seed (Hs in 0.1..0.2 m, Tp
    in 1.2..1.8 s, 64 components).  Damping zone over the last 2 m; box at x = 3 m."""
    rng = np.random.default_rng(seed)
    c = _base(nx, ny, 8.0, 4.0, 2.5)
    Hs = float(rng.uniform(0.1, 0.2))
    Tp = float(rng.uniform(1.2, 1.8))
    c["wave"] = irregular_wave(Hs, Tp, 3.3, 64, rng)
    c["damp_len"] = 2.0
    c["damp_x0"] = 6.0
    c["probe_x"] = 1.0
    c["body"] = box_body(3.0, 1.0, 0.8, 0.4, 2.5, c["rho_w"], pto_damping=0.0)
    c["solver"] = _solver(**solver_kw)
    c["dt"], c["steps"] = 5e-4, 2000
    c["name"] = f"tank {nx}x{ny} 8mx4m JONSWAP Hs={Hs:.3f} Tp={Tp:.3f} box"
    return c


def still_water(nx=64, ny=32, body=False, seed=0, **solver_kw):
    """Still water (H=0) in a 4 m x 2 m tank; optional box at its floating draft."""
    rng = np.random.default_rng(seed)
    c = _base(nx, ny, 4.0, 2.0, 1.0)
    w = regular_wave(0.0, 1.0, rng)
    c["wave"] = w
    c["damp_x0"], c["damp_len"], c["probe_x"] = 4.0, 0.0, 0.5
    c["body"] = box_body(2.0, 0.5, 0.4, 0.2, 1.0, c["rho_w"], pto_damping=0.0) if body else None
    c["solver"] = _solver(**solver_kw)
    c["dt"], c["steps"] = 1e-3, 50
    c["name"] = f"still water {nx}x{ny}"
    return c


def batch_tanks(ntanks=64, seed=0):
    """Uneven tanks: h = 1/64 m, nx in 256..768, ny in 128..256 (multiples of 64)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(ntanks):
        nx = int(rng.integers(4, 13)) * 64
        ny = int(rng.integers(2, 5)) * 64
        ny = min(ny, nx // 2)
        h = 1.0 / 64.0
        lx, ly = nx * h, ny * h
        depth = 0.5 * ly
        c = _base(nx, ny, lx, ly, depth)
        H = float(rng.uniform(0.02, 0.1))
        T = float(rng.uniform(0.8, 2.0))
        c["wave"] = regular_wave(H, T, rng)
        lam = GRAVITY * T * T / (2.0 * math.pi)
        c["damp_len"] = min(1.5 * lam, 0.25 * lx)
        c["damp_x0"] = lx - c["damp_len"]
        c["probe_x"] = 0.25
        bw = float(rng.uniform(0.25, 1.0))
        bh = float(rng.uniform(0.2, 0.6))
        c["body"] = box_body(0.5 * lx, bw, bh, 0.5 * bh, depth, c["rho_w"])
        c["solver"] = _solver(precision=1)
        c["dt"], c["steps"] = 5e-4, 500
        c["name"] = f"batch tank {k} {nx}x{ny}"
        out.append(c)
    return out


def random_fields(nx, ny, seed, scale=1.0):
    """Seeded random cell/face arrays (used to perturb states in parity tests)."""
    rng = np.random.default_rng(seed)
    return dict(
        cell=scale * rng.standard_normal((ny, nx)),
        u=scale * rng.standard_normal((ny, nx + 1)),
        v=scale * rng.standard_normal((ny + 1, nx)),
    )


def random_coefficients(nx, ny, seed, contrast=1.0):
    """Seeded positive face coefficients for Poisson tests.

    Faces on the left, right and bottom walls are zero (Neumann walls); the top
    faces are kept (Dirichlet p=0 above the top row).  ``contrast`` > 1 draws a
    log-uniform spread over that ratio.
    """
    rng = np.random.default_rng(seed)
    lo = math.log(1.0)
    hi = math.log(max(contrast, 1.0))
    bu = np.exp(rng.uniform(lo, hi, size=(ny, nx + 1))) if contrast > 1 else 0.5 + rng.uniform(size=(ny, nx + 1))
    bv = np.exp(rng.uniform(lo, hi, size=(ny + 1, nx))) if contrast > 1 else 0.5 + rng.uniform(size=(ny + 1, nx))
    bu[:, 0] = 0.0
    bu[:, nx] = 0.0
    bv[0, :] = 0.0
    return bu, bv


def unet_weights(shapes, seed):
    """Seeded He-normal weights for a list of parameter shapes (weights, then
    biases, layer by layer); biases start at zero.  Returns one flat FP32
    vector.  A weight tensor's fan-in is the product of all but its last axis."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes:
        if len(s) == 1:
            parts.append(np.zeros(s, dtype=np.float32))
        else:
            fan_in = int(np.prod(s[:-1]))
            parts.append((rng.standard_normal(s) * math.sqrt(2.0 / fan_in)).astype(np.float32))
    return np.concatenate([p.ravel() for p in parts])


def unet_dyadic_case(shapes, seed, n, h, w):
    """Seeded U-Net parameters and data on which BF16 / FP32 / FP64 arithmetic
    are all exact: one nonzero weight (+-1) per output channel of each
    convolution, head weights in {-1, 0, 1}, biases, inputs (2 channels) and
    targets in half-integer steps.  Returns (flat FP32 parameters, x, t)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes:
        if len(s) == 1:
            parts.append(rng.integers(-2, 3, size=s) * 0.5)
        elif len(s) == 2:
            parts.append(rng.choice([-1.0, 0.0, 1.0], size=s))
        else:
            W = np.zeros(s)
            kh, kw, ci, co = s
            for o in range(co):
                W[rng.integers(kh), rng.integers(kw), rng.integers(ci), o] = rng.choice([-1.0, 1.0])
            parts.append(W)
    flat = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    x = (rng.integers(-8, 9, size=(n, h, w, 2)) * 0.5).astype(np.float32)
    t = (rng.integers(-8, 9, size=(n, h, w)) * 0.5).astype(np.float32)
    return flat, x, t


def random_coefficients3(nx, ny, nz, seed, contrast=1.0):
    """Seeded positive face coefficients of the 3D pressure operator.

    Arrays (x fastest): beta_x (nz, ny, nx+1), beta_y (nz, ny+1, nx), beta_z
    (nz+1, ny, nx).  Wall and bed faces are zero (Neumann); the top faces are
    kept (Dirichlet p = 0 above the top layer).  ``contrast`` > 1 draws a
    log-uniform spread over that ratio."""
    rng = np.random.default_rng(seed)
    hi = math.log(max(contrast, 1.0))

    def draw(shape):
        return np.exp(rng.uniform(0.0, hi, size=shape)) if contrast > 1 else 0.5 + rng.uniform(size=shape)

    bx, by, bz = draw((nz, ny, nx + 1)), draw((nz, ny + 1, nx)), draw((nz + 1, ny, nx))
    bx[:, :, 0] = bx[:, :, nx] = 0.0
    by[:, 0, :] = by[:, ny, :] = 0.0
    bz[0] = 0.0
    return bx, by, bz


# Face-coefficient magnitudes of the 3D tank's pressure equation at dt = 1e-3 s
# (water, air, and the Brinkman-penalised body with kappa_p = 1e-8): the values
# the coefficient field takes in each region.
BETA3_WATER, BETA3_AIR, BETA3_BODY = 1e-3 / 1025.0, 1e-3 / 1.225, 1e-8


def poisson3d_case(nx=512, ny=256, nz=256, seed=0, lx=8.0, depth=2.0, Hs=0.2, ncomp=128, body=True):
    """Seeded coefficient field and right-hand side with the structure of the 3D
    tank's pressure equation: an 8 m x 4 m x 4 m tank (h = lx / nx), water below
    a unidirectional irregular surface (ncomp components along x with seeded
    phases and amplitudes giving a significant height ~Hs), air above, the
    coefficient blended linearly over one cell at the surface, and a vertical
    cylinder (radius 0.5 m, length 0.8 m, centred on the still-water level at
    the tank's centre) holding the body value.  Wall and bed faces are zero.
    The right-hand side is standard normal (every wavelength present).
    Returns (bx, by, bz, b) as FP64 arrays (layouts of random_coefficients3)."""
    rng = np.random.default_rng(seed)
    h = lx / nx
    ly, lz = ny * h, nz * h
    k = 2.0 * math.pi * rng.uniform(0.2, 2.0, ncomp)
    a = rng.rayleigh(1.0, ncomp)
    a *= Hs / (4.0 * math.sqrt(0.5 * np.sum(a * a)))
    ph = rng.uniform(0.0, 2.0 * math.pi, ncomp)

    def surface(x):
        return depth + np.sum(a[None, :] * np.cos(k[None, :] * x[:, None] + ph[None, :]), axis=1)

    xc, yc, zc = (np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nz) + 0.5) * h
    xf, yf, zf = np.arange(nx + 1) * h, np.arange(ny + 1) * h, np.arange(nz + 1) * h
    R, L, x0, y0 = 0.5, 0.8, 0.5 * lx, 0.5 * ly

    def field(X, Y, Z, eta):
        s = np.clip(0.5 + (Z - eta) / h, 0.0, 1.0)
        beta = (1.0 - s) * BETA3_WATER + s * BETA3_AIR
        if body:
            inside = (np.hypot(X - x0, Y - y0) < R) & (np.abs(Z - depth) < 0.5 * L)
            beta = np.where(inside, BETA3_BODY, beta)
        return beta

    Zx, Yx, Xx = np.meshgrid(zc, yc, xf, indexing="ij")
    bx = field(Xx, Yx, Zx, surface(xf)[None, None, :])
    Zy, Yy, Xy = np.meshgrid(zc, yf, xc, indexing="ij")
    by = field(Xy, Yy, Zy, surface(xc)[None, None, :])
    Zz, Yz, Xz = np.meshgrid(zf, yc, xc, indexing="ij")
    bz = field(Xz, Yz, Zz, surface(xc)[None, None, :])
    bx[:, :, 0] = bx[:, :, nx] = 0.0
    by[:, 0, :] = by[:, ny, :] = 0.0
    bz[0] = 0.0
    b = rng.standard_normal((nz, ny, nx))
    return bx, by, bz, b


def cylinder_body(xc, yc, radius, length, draft, depth, rho_w, kappa_p=1e-8, pto_damping=0.0, added_mass=0.0):
    """Vertical heaving cylinder whose mass floats it at ``draft`` (the displaced
    water mass); centred so that its bottom sits ``draft`` below still water.
    added_mass: the stabilising mass of the heave update (0: Eq. newton_u as the
    paper writes it; the cylinder's own heave added mass, ~0.9 of its mass, is
    below its mass, so the explicit force coupling is stable without it)."""
    mass = rho_w * math.pi * radius ** 2 * draft
    zc = depth - draft + 0.5 * length
    return dict(xc=xc, yc=yc, zc=zc, radius=radius, length=length, mass=mass, kappa_p=kappa_p,
                added_mass=added_mass, pto_damping=pto_damping)


def tank3d(seed=0, nx=512, ny=256, nz=256, **solver_kw):
    """The 3D tank: 8 m x 4 m x 4 m (h = lx / nx), depth 2 m, unidirectional
    JONSWAP sea along x (Hs 0.2 m, Tp 2.0 s, gamma 3.3, 128 components with
    seeded phases), a vertical cylinder of radius 0.5 m and length 0.8 m floating
    at a 0.4 m draft at the tank's centre, damping zone over the last 2 m,
    dt 1e-3 s."""
    rng = np.random.default_rng(seed)
    lx = 8.0
    h = lx / nx
    c = _base(nx, ny, lx, ny * h, 2.0)
    c["nz"], c["lz"] = nz, nz * h
    c["wave"] = irregular_wave(0.2, 2.0, 3.3, 128, rng)
    c["damp_x0"], c["damp_len"], c["probe_x"] = lx - 2.0, 2.0, 1.0
    c["body"] = cylinder_body(0.5 * lx, 0.5 * ny * h, 0.5, 0.8, 0.4, 2.0, c["rho_w"])
    c["solver"] = _solver(**solver_kw)
    c["dt"], c["steps"] = 1e-3, 500
    c["name"] = f"tank3d {nx}x{ny}x{nz} 8mx4mx4m JONSWAP cylinder"
    return c


def random_fields3(nx, ny, nz, seed, scale=1.0):
    """Seeded random cell and face arrays of a 3D grid (layouts of the 3D tank)."""
    rng = np.random.default_rng(seed)
    return dict(cell=scale * rng.standard_normal((nz, ny, nx)),
                u=scale * rng.standard_normal((nz, ny, nx + 1)),
                v=scale * rng.standard_normal((nz, ny + 1, nx)),
                w=scale * rng.standard_normal((nz + 1, ny, nx)))
