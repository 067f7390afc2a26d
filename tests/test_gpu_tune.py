"""The solver-options autotuner: it times every candidate on the caller's own
problem and returns the fastest; every candidate reaches the same FP64
tolerance (the options change the time, not the answer's tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import tune  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


def test_tank_tuner_returns_the_fastest_candidate():
    cfg = synth.tank_small(seed=1)
    cands = ((2, 2, 20), (4, 4, 8))
    best, table = tune.tune_tank(cfg, wec.PREC_MIXED, candidates=cands, steps=5, warmup=2)
    assert [(r["mg_pre"], r["mg_post"], r["restart"]) for r in table] == list(cands)
    fastest = min(table, key=lambda r: r["ms_per_step"])
    assert best == (fastest["mg_pre"], fastest["mg_post"], fastest["restart"])
    t = wec.Tank(tune.with_options(cfg, best), precision=wec.PREC_MIXED)
    r = t.step(cfg["dt"])
    assert r["residual"] <= cfg["solver"]["rtol"]
    t.close()


def test_poisson3_tuner_candidates_all_converge():
    shape = (48, 24, 32)
    bx, by, bz = synth.random_coefficients3(*shape, seed=3, contrast=1e2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    b = dev(np.random.default_rng(0).standard_normal(shape[::-1]))
    best, table = tune.tune_poisson3(shape, [dev(a) for a in (bx, by, bz)], b, wec.PREC_FP64, trials=1)
    assert len(table) == len(tune.CANDIDATES_3D)
    assert best in tune.CANDIDATES_3D
    assert all(r["iters"] > 0 for r in table)
