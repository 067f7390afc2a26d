"""Pins of the oracle's static-grid NLFK force (paper: section "Non-linear
Froude-Krylov (NLFK) forces", Eqs. p_dynamic and NLFK_p) against what physics
and the discretisation fix exactly."""
import math

import numpy as np
import pytest

from oracle import tank as O
from oracle import waves as W

RHO, G, D = 1025.0, 9.81, 0.5
REGION = (0.0, 0.0, 0.01, 200, 100)  # 2 m x 1 m, h = 1 cm, the bed at y = 0
BODY = (1.0, 0.4, 0.3)  # xc, width, height: the side walls lie on grid faces


def hydro(yc, amp=0.0):
    return O.nlfk(REGION, D, RHO, G, [amp], [2.0 * math.pi], [W.dispersion_k(2.0 * math.pi, D, G)], [0.0],
                  BODY, 0.0, yc, 1)


@pytest.mark.parametrize("yc,submerged", [(0.50, 0.15), (0.44, 0.21), (0.60, 0.05)])
def test_still_water_buoyancy_is_archimedes(yc, submerged):
    # hydrostatic pressure is linear in y, so its interpolation to psi = 0 is exact:
    # the heave force is the weight of the displaced water, the surge force zero
    fx, fy = hydro(yc)
    assert fy == pytest.approx(RHO * G * BODY[1] * submerged, rel=1e-12)
    assert abs(fx) <= 1e-9 * fy


def test_submerged_and_dry_boxes():
    fx, fy = hydro(0.2)  # fully under water: buoyancy of the whole box
    assert fy == pytest.approx(RHO * G * BODY[1] * BODY[2], rel=1e-12)
    fx, fy = hydro(0.85)  # entirely above the surface
    assert fx == 0.0 and fy == 0.0


def test_small_amplitude_fk_force_is_linear_theory():
    # a tiny regular wave: the incident pressure on the wetted bottom face at
    # height y_b above the bed is rho g a cosh(k y_b)/cosh(k d) cos(k x - w t + ph);
    # its integral over the bottom gives the linear Froude-Krylov heave force
    a, T, ph = 1e-5, 1.2, 0.7
    om = 2.0 * math.pi / T
    k = W.dispersion_k(om, D, G)
    yc = 0.5
    yb = yc - 0.5 * BODY[2]
    xl, xr = BODY[0] - 0.5 * BODY[1], BODY[0] + 0.5 * BODY[1]
    for t in (0.0, 0.31, 0.77):
        _, fy = O.nlfk(REGION, D, RHO, G, [a], [om], [k], [ph], BODY, t, yc, 0)
        ref = RHO * G * a * math.cosh(k * yb) / math.cosh(k * D) * (
            math.sin(k * xr - om * t + ph) - math.sin(k * xl - om * t + ph)) / k
        scale = RHO * G * a * BODY[1] * math.cosh(k * yb) / math.cosh(k * D)
        # midpoint sums over 1 cm cells: O((k h)^2) ~ 1e-4
        assert abs(fy - ref) <= 1e-3 * scale
    _, f0 = O.nlfk(REGION, D, RHO, G, [a], [om], [k], [ph], BODY, 0.2, yc, 0)
    _, f1 = O.nlfk(REGION, D, RHO, G, [a], [om], [k], [ph], BODY, 0.2 + 0.5 * T, yc, 0)
    assert f1 == pytest.approx(-f0, rel=1e-3)  # half a period later, the sign flips


def test_incident_pressure_is_zero_in_air():
    # a box held wholly above the crests feels nothing in either mode
    for mode in (0, 1):
        fx, fy = O.nlfk(REGION, D, RHO, G, [0.05], [5.0], [W.dispersion_k(5.0, D, G)], [0.0], BODY, 0.4, 0.9, mode)
        assert fx == 0.0 and fy == 0.0
