"""Batched tanks: one graph launch steps every tank; each tank must get exactly
the bits a stand-alone wec_step gives it, and stay on the oracle."""
import numpy as np
import pytest

from paper_2206_07732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("sigma", "u", "v", "p", "ustar", "vstar", "rhs")


@pytest.fixture(scope="module")
def wec():
    from paper_2206_07732_gb300 import build, wec as W
    build.build()
    W.load()
    return W


def uneven_cfgs():
    # different sizes (one coarsens to an odd 6x3 level), waves and seeds
    return [synth.tank_small(seed=1, nx=64, ny=32), synth.tank_small(seed=2, nx=96, ny=48),
            synth.tank_small(seed=3, nx=128, ny=64)]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_steps_match_single_tanks_bitwise(wec, prec):
    cfgs = uneven_cfgs()
    B = wec.Batch(cfgs, precision=prec)
    singles = [wec.Tank(c, precision=prec) for c in cfgs]
    dts = [c["dt"] for c in cfgs]
    pto = [0.0, 5.0, -3.0]
    for _ in range(3):
        rb = B.step(dts, pto)
        rs = [t.step(dt, f) for t, dt, f in zip(singles, dts, pto)]
        assert rb == rs
    for tb, ts in zip(B.tanks, singles):
        for name in FIELDS:
            assert np.array_equal(tb.get(name), ts.get(name)), name
    B.close()


def test_batch_tank_on_oracle(wec):
    from oracle import tank as O
    cfgs = uneven_cfgs()
    B = wec.Batch(cfgs, precision=wec.PREC_FP64)
    o = O.OracleTank(cfgs[1])
    for _ in range(2):
        rb = B.step([c["dt"] for c in cfgs])
        ro = o.step(cfgs[1]["dt"])
    g = B.tanks[1]
    for name, fo in (("sigma", O.F_SIGMA), ("u", O.F_U), ("v", O.F_V), ("p", O.F_P)):
        a, b = g.get(name), o.get(fo)
        assert np.max(np.abs(a - b)) <= 1e-10 * max(np.max(np.abs(b)), 1e-6), name
    assert rb[1]["zdot"] == pytest.approx(ro["zdot"], rel=1e-9, abs=1e-14)
    B.close()


def test_batch_step_n_records_and_launches(wec):
    cfgs = uneven_cfgs()
    B = wec.Batch(cfgs, precision=wec.PREC_MIXED)
    n0 = wec.launch_count()
    recs = B.step_n(4, [c["dt"] for c in cfgs])
    assert len(recs) == 4 * len(cfgs)
    assert all(r["status"] == 0 and r["residual"] <= 1e-8 for r in recs)
    # the step times advance per tank
    for i, c in enumerate(cfgs):
        assert recs[3 * len(cfgs) + i]["t"] == pytest.approx(4 * c["dt"])
    assert wec.launch_count() - n0 > 4 * len(cfgs) * 20
    B.close()
