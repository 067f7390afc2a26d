"""GPU parity: the CUDA library through the C ABI vs the FP64 CPU oracle.

Tolerances: FP64 path within 1e-10 relative per step (max-norm relative to the
oracle field's max), 1e-6 relative on heave after 200 steps; the pressure solver
pieces within 1e-12 (operator, V-cycle) and the solve within what rtol and the
conditioning allow.  Mixed precision: the same 1e-8 FP64 relative residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tank as O  # noqa: E402
from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402

FIELDS = [("sigma", O.F_SIGMA), ("u", O.F_U), ("v", O.F_V), ("p", O.F_P), ("ustar", O.F_USTAR),
          ("vstar", O.F_VSTAR), ("beta_u", O.F_BETA_U), ("beta_v", O.F_BETA_V), ("rhs", O.F_RHS),
          ("sigma_adv", O.F_SIGMA_ADV)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


# Absolute floors of the relative comparison (a field whose values are all
# rounding noise is compared absolutely): velocities 1e-6 m/s, pressure 1e-6 Pa,
# level set 1e-9 m, pressure right-hand side 1e-7 m^2/s, everything else 1e-300.
FLOORS = {"u": 1e-6, "v": 1e-6, "ustar": 1e-6, "vstar": 1e-6, "p": 1e-6, "sigma": 1e-9, "sigma_adv": 1e-9,
          "rhs": 1e-7}


def rel(a, b, name=None):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), FLOORS.get(name, 1e-300)))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# ------------------------------------------------------------ pressure solver --
@pytest.mark.parametrize("nx,ny,contrast", [(16, 8, 1.0), (96, 40, 1.0), (64, 32, 1e5), (256, 128, 1e3)])
def test_operator_and_vcycle_match_oracle(nx, ny, contrast):
    bu, bv = synth.random_coefficients(nx, ny, seed=nx + ny, contrast=contrast)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((ny, nx))
    P = wec.Poisson(nx, ny)
    P.set_coefficients(cuda(bu), cuda(bv))
    y = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    P.apply(cuda(x), y)
    assert rel(y.cpu().numpy(), O.poisson_apply(bu, bv, x)) < 1e-14
    z = torch.zeros_like(y)
    P.vcycle(cuda(x), z)
    zo, _ = O.vcycle(bu, bv, x)
    assert rel(z.cpu().numpy(), zo) < 1e-11


@pytest.mark.parametrize("nx,ny,contrast,rtol", [(16, 8, 1.0, 1e-13), (96, 40, 1e2, 1e-13),
                                                 (128, 64, 1e5, 1e-11), (512, 256, 1e3, 1e-12)])
def test_fgmres_solution_matches_oracle(nx, ny, contrast, rtol):
    # a log-uniform 1e5 coefficient spread has cond(A) ~ 1e9: rtol 1e-13 is below
    # what FP64 round-off lets either side reach, so that case solves to 1e-11
    bu, bv = synth.random_coefficients(nx, ny, seed=3 * nx + ny, contrast=contrast)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((ny, nx))
    P = wec.Poisson(nx, ny)
    P.set_coefficients(cuda(bu), cuda(bv))
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = P.solve(cuda(b), x, rtol=rtol)
    assert info["status"] == 0 and info["relres"] <= rtol
    xo, io = O.poisson_solve(bu, bv, b, rtol=rtol)
    assert io["status"] == 0
    assert abs(info["iters"] - io["iters"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e3 * rtol


@pytest.mark.parametrize("shift", [0, 1, 2])
@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED])
def test_bottom_split_levels_agree(shift, prec):
    # the single-CTA kernel may start at the smallest admissible level or
    # coarser (autotuned); every split computes the same V-cycle up to rounding
    nx, ny = 512, 128
    bu, bv = synth.random_coefficients(nx, ny, seed=5, contrast=1e3)
    b = np.random.default_rng(8).standard_normal((ny, nx))
    out = []
    try:
        for fused, sh in ((0, -1), (1, shift)):
            wec.set_option("mg_fused", fused)
            wec.set_option("mg_bottom_shift", sh)
            P = wec.Poisson(nx, ny, precision=prec)
            P.set_coefficients(cuda(bu), cuda(bv))
            z = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
            P.vcycle(cuda(b), z)
            out.append(z.cpu().numpy())
    finally:
        wec.set_option("mg_fused", 1)
        wec.set_option("mg_bottom_shift", -1)
    tol = 1e-12 if prec == wec.PREC_FP64 else 1e-5
    assert rel(out[1], out[0]) < tol


@pytest.mark.parametrize("nx,ny", [(96, 40), (256, 128), (288, 80), (1024, 256)])
@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED])
def test_fused_vcycle_matches_unfused(nx, ny, prec):
    # The fused tile kernels recompute halo cells with the one-pass kernels'
    # formulas; the compiler may round a fused expression differently, so the two
    # agree to rounding, and the fused V-cycle is reproducible bit for bit (a race
    # between tiles would not be).  288 x 80 has partial tiles.
    bu, bv = synth.random_coefficients(nx, ny, seed=nx * 7 + ny, contrast=1e3)
    b = np.random.default_rng(6).standard_normal((ny, nx))
    out = []
    try:
        for fused in (0, 1, 1):
            wec.set_option("mg_fused", fused)
            P = wec.Poisson(nx, ny, precision=prec)
            P.set_coefficients(cuda(bu), cuda(bv))
            z = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
            P.vcycle(cuda(b), z)
            x = torch.zeros_like(z)
            info = P.solve(cuda(b), x, rtol=1e-10)
            out.append((z.cpu().numpy(), x.cpu().numpy(), info))
    finally:
        wec.set_option("mg_fused", 1)
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
    tol = 1e-12 if prec == wec.PREC_FP64 else 1e-5
    d = rel(out[1][0], out[0][0])
    assert d < tol, d
    assert out[0][2]["status"] == out[1][2]["status"] == 0
    assert abs(out[0][2]["iters"] - out[1][2]["iters"]) <= 1
    assert rel(out[1][1], out[0][1]) < 1e3 * 1e-10
    if prec == wec.PREC_FP64:
        zo, _ = O.vcycle(bu, bv, b)
        assert rel(out[1][0], zo) < 1e-11


def test_mixed_precision_solve_reaches_fp64_tolerance():
    nx, ny = 256, 128
    bu, bv = synth.random_coefficients(nx, ny, seed=5, contrast=1e3)
    b = np.random.default_rng(3).standard_normal((ny, nx))
    P = wec.Poisson(nx, ny, precision=wec.PREC_MIXED)
    P.set_coefficients(cuda(bu), cuda(bv))
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = P.solve(cuda(b), x, rtol=1e-8)
    assert info["status"] == 0
    # the FP64 residual decides convergence: recompute it with the oracle operator
    xs = x.cpu().numpy()
    r = b - O.poisson_apply(bu, bv, xs)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * 1.0001
    xo, _ = O.poisson_solve(bu, bv, b, rtol=1e-12)
    assert rel(xs, xo) < 1e-5


def test_mixed_vcycle_is_fp32_close():
    nx, ny = 128, 64
    bu, bv = synth.random_coefficients(nx, ny, seed=9)
    b = np.random.default_rng(4).standard_normal((ny, nx))
    P = wec.Poisson(nx, ny, precision=wec.PREC_MIXED)
    P.set_coefficients(cuda(bu), cuda(bv))
    z = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    P.vcycle(cuda(b), z)
    zo, _ = O.vcycle(bu, bv, b)
    assert 1e-9 < rel(z.cpu().numpy(), zo) < 1e-4  # FP32 arithmetic, FP32-level agreement


# -------------------------------------------------------------------- step --
def _pair(cfg):
    return wec.Tank(cfg), O.OracleTank(cfg)


@pytest.mark.parametrize("case", ["small", "ragged", "nobody", "still"])
def test_initial_state_matches(case):
    cfg = {"small": synth.tank_small(seed=1), "ragged": synth.tank_small(seed=2, nx=96, ny=48),
           "nobody": synth.still_water(nx=64, ny=32, body=False),
           "still": synth.still_water(nx=64, ny=32, body=True)}[case]
    g, o = _pair(cfg)
    for name, fo in FIELDS[:4]:
        assert rel(g.get(name), o.get(fo)) < 1e-13, name


@pytest.mark.parametrize("case", ["small", "ragged", "nobody", "wave_nobody"])
def test_one_step_all_fields_match(case):
    if case == "small":
        cfg = synth.tank_small(seed=1, rtol=1e-13)
    elif case == "ragged":
        cfg = synth.tank_small(seed=2, nx=96, ny=48, rtol=1e-13)
    elif case == "nobody":
        cfg = synth.still_water(nx=64, ny=32, body=False, rtol=1e-13)
    else:
        cfg = synth.tank_small(seed=3, rtol=1e-13)
        cfg["body"] = None
    g, o = _pair(cfg)
    rg = g.step(cfg["dt"], 0.0)
    ro = o.step(cfg["dt"], 0.0)
    for name, fo in FIELDS:
        b = o.get(fo)
        if np.max(np.abs(b)) == 0.0:
            assert np.max(np.abs(g.get(name))) < 1e-12, name
            continue
        assert rel(g.get(name), b, name) < 1e-10, (name, rel(g.get(name), b, name))
    for k in ("t", "z", "zdot", "f_hydro", "f_pto"):
        assert rg[k] == pytest.approx(ro[k], rel=1e-10, abs=1e-14), k
    if not np.isnan(ro["eta_probe"]):
        assert rg["eta_probe"] == pytest.approx(ro["eta_probe"], rel=1e-10, abs=1e-14)


def test_step_from_perturbed_state_matches():
    # identical, non-trivial state on both sides (random velocities, moving body)
    cfg = synth.tank_small(seed=5, nx=64, ny=32, rtol=1e-13)
    g, o = _pair(cfg)
    rf = synth.random_fields(64, 32, seed=11, scale=0.05)
    u, v = o.get(O.F_U) + rf["u"], o.get(O.F_V) + rf["v"]
    u[:, -1] = 0.0
    v[0, :] = 0.0
    for T in (g, o):
        pass
    g.set("u", u); o.set(O.F_U, u)
    g.set("v", v); o.set(O.F_V, v)
    b = o.body()
    g.set_state(0.3, b["yc"] + 0.01, 0.05, 0.04)
    o.set_body(0.3, b["yc"] + 0.01, 0.05, 0.04)
    for _ in range(3):
        rg, ro = g.step(1e-3, 5.0), o.step(1e-3, 5.0)
        for name, fo in FIELDS[:4]:
            assert rel(g.get(name), o.get(fo)) < 1e-10, name
        assert rg["zdot"] == pytest.approx(ro["zdot"], rel=1e-10)
        # re-sync so each step starts from an identical state
        for name, fo in FIELDS[:4]:
            g.set(name, o.get(fo))
        ob = o.body()
        g.set_state(ob["t"], ob["yc"], ob["zdot"], ob["zdot_prev"])


def test_heave_after_200_steps():
    cfg = synth.tank_small(seed=0, rtol=1e-10)
    g, o = _pair(cfg)
    for n in range(200):
        rg = g.step(cfg["dt"])
        ro = o.step(cfg["dt"])
    assert rg["z"] == pytest.approx(ro["z"], rel=1e-6)
    assert rg["zdot"] == pytest.approx(ro["zdot"], rel=1e-6)
    assert rel(g.get("sigma"), o.get(O.F_SIGMA)) < 1e-6


def test_full_size_tank_one_step():
    # the large tank (1024 x 256, JONSWAP) at the size the benchmark runs
    cfg = synth.tank_large(seed=0, rtol=1e-12)
    g, o = _pair(cfg)
    for name, fo in FIELDS[:4]:
        assert rel(g.get(name), o.get(fo)) < 1e-12, name
    rg, ro = g.step(cfg["dt"]), o.step(cfg["dt"])
    for name, fo in FIELDS:
        assert rel(g.get(name), o.get(fo)) < 1e-9, name
    assert rg["zdot"] == pytest.approx(ro["zdot"], rel=1e-9)


def test_mixed_precision_step_reaches_tolerance():
    # The mixed tank computes its stencils and its multigrid preconditioner in
    # FP32 (storage, residual, Krylov basis, force and heave stay FP64).  A
    # stencil evaluation takes a few dozen FP32 operations (unit roundoff
    # 6e-8), so one step perturbs a field by ~1e-6 of its scale; 20 steps stay
    # below 1e-4.  The projection is solved to the FP64 tolerance every step.
    cfg = synth.tank_small(seed=0)
    g = wec.Tank(cfg, precision=wec.PREC_MIXED)
    o = O.OracleTank(cfg)
    for _ in range(20):
        rg = g.step(cfg["dt"])
        ro = o.step(cfg["dt"])
        assert rg["status"] == 0 and rg["residual"] <= cfg["solver"]["rtol"]
    errs = {name: rel(g.get(name), o.get(fo)) for name, fo in FIELDS[:4]}
    print("mixed vs oracle after 20 steps:", errs, "z", rg["z"], ro["z"])
    assert rg["z"] == pytest.approx(ro["z"], rel=1e-4, abs=1e-9)
    for name in ("sigma", "u", "v"):
        assert errs[name] < 1e-4, name
    assert errs["p"] < 1e-5


def test_mixed_mg_step_matches_oracle_to_solver_tolerance():
    # FP32 V-cycles only: every step stencil is FP64, so the fields differ from
    # the oracle only through the pressure solve, which both sides converge to
    # the same relative residual (rtol 1e-8, different preconditioner rounding).
    cfg = synth.tank_small(seed=0)
    g = wec.Tank(cfg, precision=wec.PREC_MIXED_MG)
    o = O.OracleTank(cfg)
    for _ in range(20):
        rg = g.step(cfg["dt"])
        ro = o.step(cfg["dt"])
        assert rg["status"] == 0 and rg["residual"] <= cfg["solver"]["rtol"]
    errs = {name: rel(g.get(name), o.get(fo)) for name, fo in FIELDS[:4]}
    print("mixed_mg vs oracle after 20 steps:", errs, "z", rg["z"], ro["z"])
    assert rg["z"] == pytest.approx(ro["z"], rel=1e-6, abs=1e-12)
    for name in ("sigma", "u", "v", "p"):
        assert errs[name] < 1e-6, name


def test_checkpoint_resume_is_bit_identical():
    cfg = synth.tank_small(seed=7, nx=64, ny=32)
    a = wec.Tank(cfg)
    for _ in range(3):
        a.step(cfg["dt"])
    blob = a.save()
    ra = [a.step(cfg["dt"]) for _ in range(3)]
    b = wec.Tank(cfg)
    b.load_state(blob)
    rb = [b.step(cfg["dt"]) for _ in range(3)]
    assert ra == rb
    for name in ("sigma", "u", "v", "p"):
        assert np.array_equal(a.get(name), b.get(name))


def test_graph_and_eager_paths_are_identical():
    # the captured graph (conditional WHILE/IF solve) and one-by-one launches run
    # the same kernels in the same order
    cfg = synth.tank_large(seed=2, nx=256, ny=64)
    a, b = wec.Tank(cfg), wec.Tank(cfg)
    b.use_graph(False)
    for _ in range(4):
        ra, rb = a.step(cfg["dt"], 3.0), b.step(cfg["dt"], 3.0)
        assert ra == rb
    for name in ("sigma", "u", "v", "p"):
        assert np.array_equal(a.get(name), b.get(name))


def test_launch_count_matches_graph_replay():
    cfg = synth.tank_small(seed=3, nx=64, ny=32)
    a, b = wec.Tank(cfg), wec.Tank(cfg)
    b.use_graph(False)
    a.step(cfg["dt"]); b.step(cfg["dt"])  # first step captures the graph
    n0 = wec.launch_count()
    ra = a.step(cfg["dt"])
    n1 = wec.launch_count()
    rb = b.step(cfg["dt"])
    n2 = wec.launch_count()
    assert ra["iters"] == rb["iters"]
    assert n1 - n0 == n2 - n1 > 50


def test_deterministic_reruns():
    cfg = synth.tank_small(seed=8, nx=64, ny=32)
    a, b = wec.Tank(cfg), wec.Tank(cfg)
    for _ in range(3):
        assert a.step(cfg["dt"]) == b.step(cfg["dt"])
    assert np.array_equal(a.get("p"), b.get("p"))


def test_pressure_solve_entry_point():
    cfg = synth.tank_small(seed=1, nx=64, ny=32, rtol=1e-12)
    g, o = _pair(cfg)
    with pytest.raises(wec.WecError):
        g.pressure_solve(torch.zeros(32, 64, dtype=torch.float64, device="cuda"),
                         torch.zeros(32, 64, dtype=torch.float64, device="cuda"), 1e-8)
    g.step(cfg["dt"])
    o.step(cfg["dt"])
    rhs = np.random.default_rng(0).standard_normal((32, 64))
    p = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    info = g.pressure_solve(cuda(rhs), p, 1e-12)
    assert info["status"] == 0
    xo, _ = O.poisson_solve(o.get(O.F_BETA_U), o.get(O.F_BETA_V), rhs, rtol=1e-12)
    assert rel(p.cpu().numpy(), xo) < 1e-8


def test_invalid_step_arguments():
    cfg = synth.tank_small(seed=1, nx=64, ny=32)
    g = wec.Tank(cfg)
    with pytest.raises(wec.WecError):
        g.step(-1.0)
    with pytest.raises(wec.WecError):
        g.set("ustar", np.zeros(g.shape("ustar")))
    with pytest.raises(wec.WecError):
        g.load_state(b"\x00" * 16)


def test_not_converged_is_reported():
    cfg = synth.tank_small(seed=1, nx=64, ny=32, rtol=1e-15)
    cfg["solver"]["max_iters"] = 1
    g = wec.Tank(cfg)
    r = g.step(cfg["dt"])
    assert r["status"] == wec.WEC_ERR_NOT_CONVERGED and r["iters"] == 1
