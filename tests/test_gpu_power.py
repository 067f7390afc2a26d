"""Power transfer from the waves to the PTO (paper, section on the power transfer
pathway): multiplying the heave equation by the heave velocity and summing over
a run, the work done by the waves, sum (F_hydro - m g) zdot dt, equals the energy
absorbed by the PTO, -sum F_PTO zdot dt, plus the change of kinetic energy.
Checked on four wave periods of the 128x64 regular-wave tank with its linear
damper, from the step records alone.  The stabilised heave update (artificial
added mass m_a, a reading of this library) adds a force m_a dt w^2 zdot in
phase with the velocity (from -m_a dt d3z/dt3): per period it supplies about
m_a dt w^2 / c of the PTO energy (16 % here), which the balance below accounts
for and checks."""
import numpy as np
import pytest

from paper_2206_07732_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    from paper_2206_07732_gb300 import build, wec
    build.build()
    wec.load()
    cfg = synth.tank_small(seed=3)
    t = wec.Tank(cfg, precision=wec.PREC_FP64)
    n = 4000  # four periods of the T = 1 s wave at dt = 1e-3
    recs = t.step_n(n, cfg["dt"])
    t.close()
    return cfg, recs


def _series(cfg, recs):
    b = cfg["body"]
    zd = np.array([0.0] + [r["zdot"] for r in recs])
    F = np.array([r["f_hydro"] for r in recs])
    Fp = np.array([r["f_pto"] for r in recs])
    mid = 0.5 * (zd[1:] + zd[:-1])
    prev = np.concatenate([[0.0], np.diff(zd)[:-1]])
    return b["mass"], b["added_mass"], cfg["g"], cfg["dt"], b["pto_damping"], zd, F, Fp, mid, prev


def test_discrete_heave_energy_identity(run):
    # the stabilised update (m + m_a)(zd1 - zd0) = dt (F - m g + F_pto) + m_a (zd0 - zdm)
    # multiplied by (zd0 + zd1) / 2 and summed: exact up to rounding
    m, ma, g, dt, c, zd, F, Fp, mid, prev = _series(*run)
    lhs = 0.5 * (m + ma) * (zd[-1] ** 2 - zd[0] ** 2)
    rhs = np.sum(dt * (F - m * g + Fp) * mid) + ma * np.sum(prev * mid)
    scale = np.sum(np.abs(dt * (F - m * g) * mid))
    assert abs(lhs - rhs) <= 1e-9 * scale


def test_wave_work_equals_absorbed_energy(run):
    # per wave period after the start-up one: W_waves = E_pto + dKE - D_stab, with
    # D_stab the work done by the stabilisation term, and D_stab / E_pto close to
    # its estimate m_a dt w^2 / c (it vanishes with dt)
    m, ma, g, dt, c, zd, F, Fp, mid, prev = _series(*run)
    P = int(round(1.0 / dt))
    est = ma * dt * (2.0 * np.pi) ** 2 / c
    for k in (1, 2, 3):
        s = slice(k * P, (k + 1) * P)
        W = np.sum(dt * (F[s] - m * g) * mid[s])
        E = -np.sum(dt * Fp[s] * mid[s])
        dKE = 0.5 * m * (zd[(k + 1) * P] ** 2 - zd[k * P] ** 2)
        D = ma * np.sum(prev[s] * mid[s]) - 0.5 * ma * (zd[(k + 1) * P] ** 2 - zd[k * P] ** 2)
        print(f"period {k}: wave work {W:.4e}, PTO {E:.4e}, dKE {dKE:.3e}, stabilisation {D:.3e} J/m, "
              f"D/E {D / E:.3f} (estimate {est:.3f})")
        assert E > 0.0  # the damper absorbs energy
        assert abs(W - (E + dKE - D)) <= 1e-6 * E
        assert 0.5 * est <= D / E <= 1.5 * est
