"""The host MPC on the 3D tank's heaving cylinder (configuration 5's "MPC-style
PTO force"): effective mass and damping from a free-decay run of the cylinder
in still water (k_h = rho_w g pi R^2), then the controller setting the PTO
force of a JONSWAP run every 0.05 s (first-order hold in between) through
wec_tank3_step: the identification is physical, the force limit holds and the
PTO absorbs energy from the waves."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import mpc  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402

SHAPE = (64, 32, 32)  # the 8 m x 4 m x 4 m tank at h = 1/8 m
DT = 2e-3


@pytest.fixture(scope="module")
def identified():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()
    c = synth.tank3d(seed=0, nx=SHAPE[0], ny=SHAPE[1], nz=SHAPE[2])
    c["wave"] = {"kind": "regular", "H": 0.0, "T": 2.0, "phase": 0.0}
    c["body"]["zc"] -= 0.02
    t = wec.Tank3(c, precision=wec.PREC_MIXED)
    recs = [t.step(DT) for _ in range(2000)]
    t.close()
    b = c["body"]
    kh = c["rho_w"] * c["g"] * math.pi * b["radius"] ** 2
    return c, kh, mpc.identify_free_decay([r["t"] for r in recs], [r["z"] - 0.02 for r in recs], kh)


def test_cylinder_free_decay_is_physical(identified):
    c, kh, (m_eff, c_r, wn, zeta) = identified
    m = c["body"]["mass"]
    print(f"cylinder free decay: m_eff {m_eff:.1f} kg (body {m:.1f}), c_r {c_r:.1f} N s/m, w_n {wn:.3f}, "
          f"zeta {zeta:.3f}")
    assert m < m_eff < 4.0 * m  # a floating cylinder's heave added mass is positive
    assert 0.0 < zeta < 0.5


def test_mpc_closed_loop_on_the_3d_tank(identified):
    _, kh, (m_eff, c_r, _, _) = identified
    c = synth.tank3d(seed=2, nx=SHAPE[0], ny=SHAPE[1], nz=SHAPE[2])
    f_max = 200.0
    Tp = c["wave"]["Tp"]
    ctl = mpc.MPC(m_eff, kh, c_r, 0.05, math.ceil(Tp / 0.05), lam1=2.0, lam2=0.2, f_max=f_max)
    amp, om, ph = wec.wave_components(c["wave"])
    kw = np.array([wec.wave_number(w, c["depth"], c["g"]) for w in om])
    xb = c["body"]["xc"]
    fexc = lambda t: kh * float(np.sum(amp * np.cos(kw * xb - om * t + ph)))
    t = wec.Tank3(c, precision=wec.PREC_MIXED)
    nsub = int(round(0.05 / DT))
    z = zd = 0.0
    F_now, E, Fmax = 0.0, [], 0.0
    for k in range(int(3 * Tp / 0.05)):
        t0 = k * 0.05
        F_next = float(ctl.solve(z, zd, F_now, fexc(t0), [fexc(t0 + (i + 1) * 0.05) for i in range(ctl.Np)])[0])
        for f in ctl.ramp(F_now, F_next, nsub):
            r = t.step(DT, f)
            assert r["status"] == 0
            E.append(-f * 0.5 * (zd + r["zdot"]) * DT)
            zd = r["zdot"]
            Fmax = max(Fmax, abs(r["f_pto"]))
        z = r["z"]
        F_now = F_next
    t.close()
    n1 = int(Tp / DT)
    absorbed = float(np.sum(E[n1:]))
    print(f"3D closed loop: absorbed {absorbed:.4f} J over the last two peak periods, max |F_PTO| {Fmax:.2f} N")
    assert Fmax <= f_max * (1 + 1e-9)
    assert absorbed > 0.0
