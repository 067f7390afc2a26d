"""Edge cases of the step and the solver against the oracle: the smallest
admissible tank, the extremes of every solver option, a zero right-hand side,
a solve far larger than the benchmark grid (checked by its FP64 residual, which
holds at any size), and a batch of one tank."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tank as O  # noqa: E402
from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402

FIELDS = [("sigma", O.F_SIGMA), ("u", O.F_U), ("v", O.F_V), ("p", O.F_P), ("ustar", O.F_USTAR),
          ("vstar", O.F_VSTAR), ("rhs", O.F_RHS)]
FLOORS = {"u": 1e-6, "v": 1e-6, "ustar": 1e-6, "vstar": 1e-6, "p": 1e-6, "sigma": 1e-9, "rhs": 1e-7}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


def rel(a, b, name):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), FLOORS.get(name, 1e-300)))


def one_step_matches(cfg, steps=1):
    g, o = wec.Tank(cfg), O.OracleTank(cfg)
    for _ in range(steps):
        rg = g.step(cfg["dt"], 0.0)
        ro = o.step(cfg["dt"], 0.0)
    for name, fo in FIELDS:
        assert rel(g.get(name), o.get(fo), name) < 1e-10, name
    for k in ("z", "zdot", "f_hydro"):
        assert rg[k] == pytest.approx(ro[k], rel=1e-10, abs=1e-14), k
    assert rg["iters"] == ro["iters"]
    g.close()


def test_smallest_admissible_tank():
    # 16 x 8 cells (h = 0.25 m, the box two cells wide): every multigrid level
    # lies inside the single-CTA bottom kernel
    one_step_matches(synth.tank_small(seed=5, nx=16, ny=8, rtol=1e-13), steps=3)


@pytest.mark.parametrize("opts", [dict(n_reinit=0, n_jacobi=1, mg_pre=1, mg_post=0, restart=20),
                                  dict(n_reinit=0, n_jacobi=1, mg_pre=1, mg_post=1, restart=1),
                                  dict(n_reinit=4, n_jacobi=4, mg_pre=4, mg_post=4, restart=32),
                                  dict(n_reinit=2, n_jacobi=2, mg_pre=3, mg_post=1, restart=5)])
def test_option_extremes(opts):
    # no reinitialisation and one Jacobi sweep; V(1,0); restart 1; the largest
    # tile halo (8 cells, V(4,4)) with the longest basis (32)
    cfg = synth.tank_small(seed=6, nx=64, ny=32, rtol=1e-10)
    cfg["solver"].update(opts)
    one_step_matches(cfg, steps=2)


def test_iteration_cap():
    # FGMRES(1) preconditioned by V(1,0) stagnates on this operator; both sides
    # stop at the cap with the same iterate
    cfg = synth.tank_small(seed=6, nx=64, ny=32, rtol=1e-10)
    cfg["solver"].update(n_reinit=0, n_jacobi=1, mg_pre=1, mg_post=0, restart=1, max_iters=50)
    o = O.OracleTank(cfg)
    assert o.step(cfg["dt"], 0.0)["status"] == wec.WEC_ERR_NOT_CONVERGED
    one_step_matches(cfg, steps=1)


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED])
def test_zero_right_hand_side(prec):
    nx, ny = 64, 32
    bu, bv = synth.random_coefficients(nx, ny, seed=1, contrast=1e3)
    P = wec.Poisson(nx, ny, precision=prec)
    P.set_coefficients(torch.from_numpy(bu).cuda(), torch.from_numpy(bv).cuda())
    x = torch.full((ny, nx), 3.0, dtype=torch.float64, device="cuda")
    info = P.solve(torch.zeros(ny, nx, dtype=torch.float64, device="cuda"), x, rtol=1e-8)
    assert info["status"] == 0 and info["iters"] == 0
    assert float(x.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [wec.PREC_FP64, wec.PREC_MIXED])
def test_large_solve_reaches_tolerance(prec):
    # 2048 x 512 (1 M cells, 4x the benchmark grid), density contrast 1e3: the
    # FP64 residual recomputed by the oracle's operator meets rtol
    nx, ny = 2048, 512
    bu, bv = synth.random_coefficients(nx, ny, seed=9, contrast=1e3)
    b = np.random.default_rng(9).standard_normal((ny, nx))
    P = wec.Poisson(nx, ny, precision=prec)
    P.set_coefficients(torch.from_numpy(bu).cuda(), torch.from_numpy(bv).cuda())
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = P.solve(torch.from_numpy(b).cuda(), x, rtol=1e-8)
    assert info["status"] == 0
    r = b - O.poisson_apply(bu, bv, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(b)


def test_batch_of_one_tank():
    cfg = synth.tank_small(seed=7, nx=64, ny=32)
    Bt = wec.Batch([cfg], precision=wec.PREC_FP64)
    t = wec.Tank(cfg, precision=wec.PREC_FP64)
    for _ in range(3):
        assert Bt.step([cfg["dt"]]) == [t.step(cfg["dt"])]
    assert np.array_equal(Bt.tanks[0].get("p"), t.get("p"))
    Bt.close()
