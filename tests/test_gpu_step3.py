"""The 3D tank step on the GPU (wec_tank3_step) against the 3D step oracle:
the initial state, every field after each step (FP64, 1e-10 relative per step),
the heave after 200 steps (1e-6 relative), the FP32-V-cycle path's error, and
the 512 x 256 x 256 tank: by its properties (solve residual, divergence, finite
heave) and, for one step, every field against the oracle's step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tank3d as T3  # noqa: E402
from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


FIELDS = ((wec.F3_SIGMA, T3.F_SIGMA, "sigma"), (wec.F3_U, T3.F_U, "u"), (wec.F3_V, T3.F_V, "v"),
          (wec.F3_W, T3.F_W, "w"), (wec.F3_P, T3.F_P, "p"))


def rel(a, b, floor=1e-300):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


def _cfg(nx, ny, nz, seed=1, rtol=1e-12, **kw):
    c = synth.tank3d(seed=seed, nx=nx, ny=ny, nz=nz, rtol=rtol, **kw)
    return c


@pytest.mark.parametrize("shape", [(32, 8, 16), (40, 12, 20)])
def test_initial_state_matches_oracle(shape):
    c = _cfg(*shape)
    t, o = wec.Tank3(c), T3.OracleTank3(c)
    for fg, fo, name in FIELDS:
        assert rel(t.get(fg), o.get(fo), 1e-12) < 1e-12, name
    t.close()


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED_DF])
@pytest.mark.parametrize("shape,body", [((32, 8, 16), True), ((40, 12, 20), True), ((24, 8, 16), False)])
def test_steps_match_oracle(shape, body, prec):
    # FP64 stencils, and double-float stencils (FP32 pairs) with FP32 V-cycles:
    # both hold every field within 1e-10 of the FP64 oracle step after step
    c = _cfg(*shape)
    if not body:
        c["body"] = None
    t, o = wec.Tank3(c, precision=prec), T3.OracleTank3(c)
    for s in range(4):
        r, ro = t.step(c["dt"]), o.step(c["dt"])
        assert r["status"] == 0 and ro["status"] == 0
        # v is identically zero in the oracle when nothing breaks the y-symmetry:
        # its error is measured against the velocity scale max|u|
        vs = np.max(np.abs(o.get(T3.F_U)))
        errs = {name: rel(t.get(fg), o.get(fo), vs if name == "v" else 1e-12) for fg, fo, name in FIELDS}
        print(f"{shape} step {s}: {errs} F {r['f_hydro']:.6f} / {ro['f_hydro']:.6f} its {r['iters']}/{ro['iters']}")
        for name, e in errs.items():
            assert e < 1e-10, (s, name, e)
        if body:
            assert r["f_hydro"] == pytest.approx(ro["f_hydro"], rel=1e-10)
            assert r["zdot"] == pytest.approx(ro["zdot"], rel=1e-10, abs=1e-14)
        if prec == wec.PREC_FP64:  # the same preconditioner as the oracle's
            assert abs(r["iters"] - ro["iters"]) <= 1
    t.close()


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED_DF, wec.PREC_MIXED])
@pytest.mark.parametrize("shape", [(40, 12, 20), (48, 16, 16)])
def test_momentum_kernel_forms_agree(shape, prec):
    # the momentum system as one kernel or two ("tank3_split_momentum"): the
    # same per-face arithmetic -- the same bits in float pairs, whose products
    # and sums are explicit; in FP64 and FP32 the compiler may contract a
    # product into a sum differently in each kernel, so there the fields agree
    # to rounding
    c = _cfg(*shape)
    out = []
    try:
        for split in (1, 0):
            wec.set_option("tank3_split_momentum", split)
            t = wec.Tank3(c, precision=prec)
            for _ in range(3):
                assert t.step(c["dt"])["status"] == 0
            out.append([t.get(fg) for fg, _, _ in FIELDS])
            t.close()
    finally:
        wec.set_option("tank3_split_momentum", 1)
    tol = {wec.PREC_MIXED_DF: 0.0, wec.PREC_FP64: 1e-12, wec.PREC_MIXED: 1e-5}[prec]
    for form, fields in enumerate(out[1:], 1):
        for (_, _, name), a, b in zip(FIELDS, fields, out[0]):
            e = rel(a, b, 1e-12)
            print(f"{shape} prec {prec} form {form} {name}: {e:.2e}")
            assert e <= tol, (form, name, e)


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED_DF])
@pytest.mark.parametrize("ncyc", [2, 3])
def test_fixed_point_cycles_match_oracle(prec, ncyc):
    # n_cycles > 1 (section "Time stepping scheme"): force on the iterate, heave
    # from level n, sigma^n advected with the means of levels n and n+1,k, level
    # n's momentum system; every field within 1e-10 of the oracle's cycles
    c = _cfg(40, 12, 20, seed=7)
    c["solver"]["n_cycles"] = ncyc
    t, o = wec.Tank3(c, precision=prec), T3.OracleTank3(c)
    for s in range(3):
        r, ro = t.step(c["dt"]), o.step(c["dt"])
        assert r["status"] == 0 and ro["status"] == 0
        vs = np.max(np.abs(o.get(T3.F_U)))
        errs = {name: rel(t.get(fg), o.get(fo), vs if name == "v" else 1e-12) for fg, fo, name in FIELDS}
        print(f"{ncyc} cycles, step {s}: {errs}, F {r['f_hydro']:.6f} / {ro['f_hydro']:.6f}")
        for name, e in errs.items():
            assert e < 1e-10, (s, name, e)
        assert r["f_hydro"] == pytest.approx(ro["f_hydro"], rel=1e-10)
        assert r["zdot"] == pytest.approx(ro["zdot"], rel=1e-10, abs=1e-14)
    t.close()


def test_cycle_options_are_checked():
    c = _cfg(16, 8, 8)
    c["solver"]["n_cycles"] = 9
    with pytest.raises(wec.WecError):
        wec.Tank3(c)


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED_DF])
def test_heave_after_200_steps(prec):
    c = _cfg(32, 8, 16, seed=3, rtol=1e-10)
    t, o = wec.Tank3(c, precision=prec), T3.OracleTank3(c)
    for _ in range(200):
        r, ro = t.step(c["dt"]), o.step(c["dt"])
    print(f"200 steps: z {r['z']:.9e} / {ro['z']:.9e}, zdot {r['zdot']:.9e} / {ro['zdot']:.9e}")
    assert r["z"] == pytest.approx(ro["z"], rel=1e-6)
    assert r["zdot"] == pytest.approx(ro["zdot"], rel=1e-6)
    t.close()


def test_fp32_vcycle_path_error_against_the_oracle():
    # FP32 V-cycles inside the FP64 FGMRES: every solve reaches the same FP64
    # residual; the fields differ from the oracle by what rtol allows
    c = _cfg(32, 8, 16, seed=4, rtol=1e-8)
    t, o = wec.Tank3(c, precision=wec.PREC_MIXED_MG), T3.OracleTank3(c)
    for _ in range(10):
        r, ro = t.step(c["dt"]), o.step(c["dt"])
        assert r["status"] == 0 and r["residual"] <= 1e-8
    errs = {name: rel(t.get(fg), o.get(fo), 1e-12) for fg, fo, name in FIELDS}
    print(f"FP32 V-cycles, 10 steps: {errs}, heave {abs(r['z'] - ro['z']) / abs(ro['z']):.2e}")
    assert max(errs.values()) < 1e-5
    t.close()


def test_fp32_stencil_path_error_against_the_oracle():
    # WEC_PREC_MIXED: the step's stencils in FP32 over FP32 working copies, the
    # force, heave, solve and projection FP64; the error against the FP64 oracle
    # after 20 steps is of FP32 size (stated, bounded by 1e-4)
    c = _cfg(32, 8, 16, seed=6, rtol=1e-8)
    t, o = wec.Tank3(c, precision=wec.PREC_MIXED), T3.OracleTank3(c)
    for _ in range(20):
        r, ro = t.step(c["dt"]), o.step(c["dt"])
        assert r["status"] == 0 and r["residual"] <= 1e-8
    vs = np.max(np.abs(o.get(T3.F_U)))
    errs = {name: rel(t.get(fg), o.get(fo), vs if name == "v" else 1e-12) for fg, fo, name in FIELDS}
    hz = abs(r["z"] - ro["z"]) / abs(ro["z"])
    print(f"FP32 stencils, 20 steps: {errs}, heave {hz:.2e}")
    assert max(errs.values()) < 1e-4
    assert hz < 1e-4


def test_full_size_tank_step():
    c = synth.tank3d(seed=0)
    t = wec.Tank3(c)
    rs = []
    for _ in range(2):
        r = t.step(c["dt"])
        assert r["status"] == 0
        assert r["residual"] <= c["solver"]["rtol"]
        assert np.isfinite(r["f_hydro"]) and np.isfinite(r["zdot"])
        rs.append(r)
    # the first step's force is the initial hydrostatic pressure's: the weight of
    # the floating cylinder times (1 + eta / draft) with the incident wave at the
    # body (|eta| well below the 0.4 m draft); the second carries the impulsive
    # pressure that brings the Airy flow through the body to rest
    b = c["body"]
    ratio = rs[0]["f_hydro"] / (b["mass"] * c["g"])
    print(f"512x256x256: {[q['iters'] for q in rs]} iterations, first-step F / mg {ratio:.4f}, "
          f"div {rs[-1]['div_norm']:.3e}")
    assert 0.5 < ratio < 1.5
    t.close()


def test_full_size_step_matches_the_oracle_everywhere():
    # One step of the 512 x 256 x 256 tank of configuration 5 from its initial
    # state: every cell and face of sigma, u, v, w and p against the oracle's step
    # (run on all host cores), for the FP64 path and the FP32-V-cycle path, both
    # sides solving to 1e-12.  The comparison covers the interior fast path of
    # the momentum and Jacobi stencils (32-bit offsets, no ghost rules), every
    # boundary face, and the cell layers of the force integral around the cylinder.
    from paper_2206_07732_gb300 import tune
    c = tune.with_options(synth.tank3d(seed=0, rtol=1e-12), (3, 3, 5))
    o = T3.OracleTank3(c)
    ro = o.step(c["dt"])
    assert ro["status"] == 0
    ref = {name: o.get(fo) for _, fo, name in FIELDS}
    del o
    vs = np.max(np.abs(ref["u"]))
    for prec, bound in ((wec.PREC_FP64, 1e-10), (wec.PREC_MIXED_MG, 1e-9), (wec.PREC_MIXED_DF, 1e-9)):
        t = wec.Tank3(c, precision=prec)
        r = t.step(c["dt"])
        assert r["status"] == 0 and r["residual"] <= 1e-12
        errs = {name: rel(t.get(fg), ref[name], vs if name == "v" else 1e-12) for fg, _, name in FIELDS}
        t.close()
        print(f"512x256x256 step, precision {prec}: {errs}, F {r['f_hydro']:.9f} / {ro['f_hydro']:.9f}, "
              f"its {r['iters']} / {ro['iters']}")
        for name, e in errs.items():
            assert e < bound, (prec, name, e)
        assert r["f_hydro"] == pytest.approx(ro["f_hydro"], rel=1e-10)
        assert r["zdot"] == pytest.approx(ro["zdot"], rel=1e-10, abs=1e-14)


def test_invalid_step_uses():
    c = _cfg(16, 8, 8)
    t = wec.Tank3(c, step=False)
    with pytest.raises(wec.WecError):  # created without solver options
        t.step(c["dt"])
    t.close()
    t = wec.Tank3(c)
    with pytest.raises(wec.WecError):
        t.step(0.0)
    t.close()
