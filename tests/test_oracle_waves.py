"""Pins of the oracle's wave utilities against what the paper and mathematics fix.

Section "Regular waves" (Eqs. dispersion_relation, explicit_dispersion_relation,
group_velocity, regular_wave_power, deep_water_limit) and Section "Irregular
waves" (Eqs. irregular_elevation, wave_spectrum_amplitude, Bretshneider_wave_spec).
"""
import math
import os

import numpy as np
import pytest

from oracle import waves as W

G = 9.81


def _read_golden(golden_dir, name):
    out = {}
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


@pytest.mark.parametrize("depth", [0.05, 0.5, 1.0, 2.5, 40.0])
def test_dispersion_residual(depth):
    for w in np.linspace(0.2, 25.0, 50):
        k = W.dispersion_k(w, depth, G)
        assert abs(G * k * math.tanh(k * depth) - w * w) <= 1e-13 * w * w


def test_dispersion_limits():
    # deep water: omega^2 = g k (Eq. deep_water_limit)
    w = 20.0
    assert W.dispersion_k(w, 50.0, G) == pytest.approx(w * w / G, rel=1e-14)
    # shallow water: k -> omega / sqrt(g d)
    w, d = 0.01, 0.5
    assert W.dispersion_k(w, d, G) == pytest.approx(w / math.sqrt(G * d), rel=1e-5)


def test_fenton_close_to_exact():
    # Fenton's explicit form is an approximation "accurate enough for practical
    # purposes at all water depths": measured max relative error ~5e-4.
    worst = 0.0
    for d in (0.1, 0.5, 1.0, 2.5, 10.0):
        for w in np.linspace(0.3, 25.0, 60):
            kd = W.dispersion_k(w, d, G) * d
            worst = max(worst, abs(W.fenton_kd(w, d, G) - kd) / kd)
    assert worst < 1e-3
    assert worst > 1e-6  # it is an approximation, not the exact root


def test_deep_water_power(golden_dir):
    gold = _read_golden(golden_dir, "deep_water_power.txt")
    rho = 1025.0
    # rho g^2 / (32 pi) ~ 1e3: P ~ H^2 T kW/m in deep water
    assert rho * G * G / (32.0 * math.pi) / 1000.0 == pytest.approx(gold["factor_regular_kW"], rel=0.03)
    H, T, d = 0.1, 1.0, 100.0
    w = 2 * math.pi / T
    k = W.dispersion_k(w, d, G)
    P = W.regular_wave_power(H, w, k, d, rho, G)
    assert P == pytest.approx(rho * G * G * H * H * T / (32 * math.pi), rel=1e-10)
    # deep water group velocity is half the phase velocity
    assert W.group_velocity(w, k, d) == pytest.approx(0.5 * w / k, rel=1e-12)


def test_bretschneider_zeroth_moment():
    # int_0^inf A w^-5 exp(-B w^-4) dw = A / (4 B) = 173 / (4 692) Hs^2 = Hs^2 / 16
    from scipy.integrate import quad
    for T in (0.8, 1.6, 2.5):
        m0 = quad(lambda w: W.bretschneider_printed(w, 0.15, T), 0, np.inf, limit=200)[0]
        assert m0 == pytest.approx(0.15 ** 2 / 16.0, rel=1e-9)


def test_bretschneider_peak_matches_caption(golden_dir):
    gold = _read_golden(golden_dir, "bretschneider_caption.txt")
    wp = 2 * math.pi / gold["Tp"]
    assert wp == pytest.approx(gold["omega_p"], abs=5e-5)
    e = 1e-5
    S = lambda w: float(W.bretschneider(w, gold["Hs"], gold["Tp"]))
    dS = (S(wp + e) - S(wp - e)) / (2 * e)
    assert abs(dS) < 1e-9 * S(wp)
    assert S(wp) > S(0.95 * wp) and S(wp) > S(1.05 * wp)
    # the printed form with T = Tp peaks elsewhere -- the reading fixes that
    T1 = W.bretschneider_period(gold["Tp"])
    assert T1 / gold["Tp"] == pytest.approx(0.772, abs=1e-3)


def test_jonswap_reduces_and_enhances():
    w = np.linspace(1.0, 20.0, 400)
    Hs, Tp = 0.15, 1.6
    np.testing.assert_allclose(W.jonswap(w, Hs, Tp, 1.0), W.bretschneider(w, Hs, Tp), rtol=1e-15)
    wp = 2 * math.pi / Tp
    assert float(W.jonswap(wp, Hs, Tp, 3.3) / W.bretschneider(wp, Hs, Tp)) == pytest.approx(3.3, rel=1e-14)


def test_jonswap_components_hs_and_band(golden_dir):
    band = _read_golden(golden_dir, "temporal_band.txt")
    assert W.BAND_LO == pytest.approx(band["omega_lo"] / band["omega_p"], abs=2e-3)
    assert W.BAND_HI == pytest.approx(band["omega_hi"] / band["omega_p"], abs=2e-3)
    rng = np.random.default_rng(1)
    ph = rng.uniform(0, 2 * math.pi, 64)
    a, w, p = W.jonswap_components(0.15, 1.6, 3.3, 64, ph)
    assert 4.0 * math.sqrt(np.sum(a * a) / 2.0) == pytest.approx(0.15, rel=1e-14)
    dw = w[1] - w[0]
    np.testing.assert_allclose(np.diff(w), dw, rtol=1e-12)
    # Eq. wave_spectrum_amplitude before the Hs normalisation
    a0, _, _ = W.jonswap_components(0.15, 1.6, 3.3, 64, ph, normalise=False)
    np.testing.assert_allclose(a0 ** 2 / (2 * dw), W.jonswap(w, 0.15, 1.6, 3.3), rtol=1e-13)
    # gamma = 3.3 carries more energy than Bretschneider at the same Hs; the
    # normalisation undoes it.  The factor matches the usual JONSWAP estimate
    # 1 / (1 - 0.287 ln gamma) within a few percent.
    ratio = float(np.sum(a0 ** 2) / np.sum(a ** 2))
    assert ratio == pytest.approx(1.0 / (1.0 - 0.287 * math.log(3.3)), rel=0.03)
    # with gamma = 1 truncating the band loses only a little energy
    b0, _, _ = W.jonswap_components(0.15, 1.6, 1.0, 64, ph, normalise=False)
    assert 0.95 < float(np.sum(b0 ** 2)) / (2.0 * 0.15 ** 2 / 16.0) <= 1.0
