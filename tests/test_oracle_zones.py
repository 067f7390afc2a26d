"""Pins of the oracle's wave-damping zone and top vorticity-damping layer
(section "Numerical wave tank": a relaxation zone of the Jacobsen kind at the
outlet, Eq. spongelayer at the top), checked against weights worked out by
hand at a few positions -- not by calling the oracle's own weight functions.

Damping zone (outlet, last 1 m of the 4 m tank): alpha(xi) = (e^{xi^3.5} - 1)/(e - 1)
with xi the distance into the zone over its length.  Worked values:
  xi = 0.515625: xi^3.5 = 0.098419..., alpha = 0.10343.../1.71828... = 0.0602040436
  xi = 0.5     : xi^3.5 = 0.0883883..., alpha = 0.0924134.../1.71828... = 0.0537817917
  xi = 0.9375  : xi^3.5 = 0.7980..., alpha = 1.22067.../1.71828... = 0.7104028415
The level set is blended toward still water, sigma <- (1 - alpha) sigma + alpha (y - d),
so a uniform offset eps decays to (1 - alpha) eps per call; the momentum gets
alpha rho/dt on its diagonal, so a uniform current U0 in still water predicts
U0 / (1 + alpha).

Vorticity damping over the top four cells: g = rho_a (cos(pi z~) + 1) / (4 dt),
z~ = (y - y_top) / (4 h).  A uniform current U0 in the air predicts
U0 / (1 + (cos(pi z~) + 1) / 4); at the u-faces of the top four cell rows
z~ = -1/8, -3/8, -5/8, -7/8 give 0.6752331775, 0.7431237691, 0.8663040408,
0.9813252655, and 1 below them.
"""
import numpy as np
import pytest

from oracle import tank as O
from paper_2206_07732_gb300 import synth

ALPHA = {0.515625: 0.0602040436, 0.5: 0.0537817917, 0.9375: 0.7104028415}
TOP = [0.6752331775, 0.7431237691, 0.8663040408, 0.9813252655]


def _still_tank(nx=128, ny=64):
    c = synth.tank_small(seed=0, nx=nx, ny=ny)
    c["wave"] = dict(kind="regular", H=0.0, T=1.0, phase=0.0)
    c["body"] = None
    return c


def test_damping_zone_blends_sigma_with_the_jacobsen_weight():
    c = _still_tank()
    T = O.OracleTank(c)
    h = c["lx"] / c["nx"]
    x = (np.arange(c["nx"]) + 0.5) * h
    y = (np.arange(c["ny"]) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    eps = 0.01
    T.set(O.F_SIGMA, Y - c["depth"] + eps)
    T.set(O.F_U, np.zeros(T.shape(O.F_U)))
    T.set(O.F_V, np.zeros(T.shape(O.F_V)))
    ncalls = 3
    for _ in range(ncalls):
        T.advect(1e-3)
    ratio = (T.get(O.F_SIGMA) - (Y - c["depth"])) / eps
    # column of the cell centre at xi = 0.515625 (x = 3.515625 m)
    i = int(round(3.515625 / h - 0.5))
    np.testing.assert_allclose(ratio[:, i], (1.0 - ALPHA[0.515625]) ** ncalls, rtol=1e-9)
    # outside the zone the offset is untouched (zero velocity: no advection)
    assert np.allclose(ratio[:, : int(3.0 / h) - 1], 1.0, rtol=0, atol=1e-12)
    # the last column, xi = 0.984375 > 0.9375: at least as damped as the worked value there
    assert np.all(ratio[:, -1] < (1.0 - ALPHA[0.9375]) ** ncalls + 1e-12)


def test_damping_zone_momentum_weight_on_a_uniform_current():
    c = _still_tank()
    T = O.OracleTank(c)
    h = c["lx"] / c["nx"]
    U0 = 0.05
    T.set(O.F_U, np.full(T.shape(O.F_U), U0))
    T.set(O.F_V, np.zeros(T.shape(O.F_V)))
    T.step(1e-3)
    us = T.get(O.F_USTAR)
    j = int(0.5 * c["depth"] / h)  # mid-depth row of u-faces, water only
    for x, a in ((3.5, ALPHA[0.5]), (3.9375, ALPHA[0.9375])):
        i = int(round(x / h))  # the u-face at x = i h
        assert us[j, i] / U0 == pytest.approx(1.0 / (1.0 + a), rel=1e-4)
    # a face outside the zone (x = 2 m) keeps the current
    assert us[j, int(round(2.0 / h))] / U0 == pytest.approx(1.0, rel=1e-4)


def test_vorticity_damping_layer_on_a_uniform_current_in_the_air():
    c = _still_tank()
    T = O.OracleTank(c)
    h = c["lx"] / c["nx"]
    U0 = 0.05
    T.set(O.F_U, np.full(T.shape(O.F_U), U0))
    T.set(O.F_V, np.zeros(T.shape(O.F_V)))
    T.step(1e-3)
    us = T.get(O.F_USTAR)
    i = int(round(1.5 / h))  # mid-tank, away from the inflow and the damping zone
    ny = c["ny"]
    for m, f in enumerate(TOP):  # rows ny-1, ny-2, ny-3, ny-4
        assert us[ny - 1 - m, i] / U0 == pytest.approx(f, rel=2e-4)
    # below the layer the air keeps the current
    assert us[ny - 6, i] / U0 == pytest.approx(1.0, rel=2e-4)
