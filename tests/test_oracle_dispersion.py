"""In-tank dispersion pin (section "Numerical wave tank", Eq. dispersion_relation):
the oracle's tank of configuration 1 without the body carries its generated
linear wave (H 0.05 m, T 1 s, depth 1 m) at the celerity omega / kappa that
omega^2 = g kappa tanh(kappa d) fixes, measured between two probes at x = 1 m
and x = 2 m from the phase of the surface elevation there over one period
(least-squares fit of a cos + b sin + c at the wave's frequency; the surface
is the level set's zero crossing in the probe column, interpolated between
the two nearest columns).  Within 3 % at 128 x 64, the error shrinking from
64 x 32 to 128 x 64 to 256 x 128 (measured: -3.3 %, -2.1 %, -1.9 %).  kappa
comes from the closed form checked in test_oracle_waves (Newton on the
dispersion relation)."""
import math

import numpy as np
import pytest

from oracle import tank as O
from oracle import waves as OW
from paper_2206_07732_gb300 import synth

X1, X2, TEND, DT = 1.0, 2.0, 1.0, 1e-3


def _eta_column(s, i, h, depth):
    col = s[:, i]
    for j in range(len(col) - 1):
        if col[j] < 0.0 <= col[j + 1]:
            return (j + 0.5) * h + h * col[j] / (col[j] - col[j + 1]) - depth
    return float("nan")


def _celerity(nx, ny):
    c = synth.tank_small(seed=0, nx=nx, ny=ny)
    c["body"] = None
    T = O.OracleTank(c)
    h = c["lx"] / nx

    def eta_x(s, x):
        f = x / h - 0.5
        i = int(math.floor(f))
        w = f - i
        return (1 - w) * _eta_column(s, i, h, c["depth"]) + w * _eta_column(s, i + 1, h, c["depth"])

    n = int(round(TEND / DT))
    ts, e1, e2 = np.zeros(n), np.zeros(n), np.zeros(n)
    for k in range(n):
        T.step(DT)
        s = T.get(O.F_SIGMA)
        ts[k], e1[k], e2[k] = (k + 1) * DT, eta_x(s, X1), eta_x(s, X2)
    om = 2.0 * math.pi / c["wave"]["T"]
    kap = OW.dispersion_k(om, c["depth"], c["g"])
    A = np.stack([np.cos(om * ts), np.sin(om * ts), np.ones_like(ts)], 1)
    p1 = np.linalg.lstsq(A, e1, rcond=None)[0]
    p2 = np.linalg.lstsq(A, e2, rcond=None)[0]
    # eta = a cos(kappa x - omega t + theta): the phase of the fit grows by kappa (x2 - x1)
    d = (math.atan2(p2[1], p2[0]) - math.atan2(p1[1], p1[0])) % (2.0 * math.pi)
    lam = 2.0 * math.pi / kap
    whole = round((X2 - X1) / lam - d / (2.0 * math.pi))
    k_num = (d + 2.0 * math.pi * whole) / (X2 - X1)
    amp = (math.hypot(p1[0], p1[1]), math.hypot(p2[0], p2[1]))
    return om / k_num, om / kap, amp


@pytest.fixture(scope="module")
def celerities():
    return {n: _celerity(n, n // 2) for n in (64, 128, 256)}


def test_generated_wave_travels_at_the_dispersion_celerity(celerities):
    c_num, c_th, amp = celerities[128]
    assert abs(c_num / c_th - 1.0) < 0.03
    # the probes see the generated wave (H / 2 = 0.025 m), not noise
    assert 0.015 < amp[0] < 0.035 and 0.015 < amp[1] < 0.035


def test_celerity_error_shrinks_under_refinement(celerities):
    e = [abs(celerities[n][0] / celerities[n][1] - 1.0) for n in (64, 128, 256)]
    assert e[0] > e[1] > e[2]
