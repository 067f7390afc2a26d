"""Oracle wave utilities (plain numpy, FP64) -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use anything under ``oracle/``.  The product path never does.

Implements, from the paper's Section "Regular waves" / "Irregular waves":
  * linear dispersion omega^2 = g k tanh(k d)           (Eq. dispersion_relation)
  * Fenton's explicit approximation of k d               (Eq. explicit_dispersion_relation)
  * group velocity and regular-wave power                (Eqs. group_velocity, regular_wave_power)
  * component amplitude a_i = sqrt(2 S(omega_i) d omega) (Eq. wave_spectrum_amplitude)
  * Bretschneider spectrum                               (Eq. Bretshneider_wave_spec)
  * JONSWAP = Bretschneider x peak enhancement gamma^r   (not in the paper; the workload asks
    for it -- standard Hasselmann et al. form, s = 0.07 / 0.09)
"""
from __future__ import annotations

import math

import numpy as np

# Band of the discretised spectrum as multiples of the peak frequency.  The
# paper's irregular-wave study spans 1.6 - 20 rad/s around omega_p = 3.5955
# rad/s (Section "Temporal resolution"), i.e. 0.445 - 5.56 omega_p.
BAND_LO = 1.6 / 3.5955
BAND_HI = 20.0 / 3.5955


def dispersion_k(omega, depth, g):
    """Wavenumber solving omega^2 = g k tanh(k d) (Eq. dispersion_relation) by Newton."""
    omega = float(omega)
    if omega == 0.0:
        return 0.0
    k = max(omega * omega / g, omega / math.sqrt(g * depth))
    for _ in range(100):
        th = math.tanh(k * depth)
        f = g * k * th - omega * omega
        df = g * th + g * k * depth * (1.0 - th * th)
        dk = f / df
        k -= dk
        if abs(dk) <= 1e-16 * k:
            break
    return k


def fenton_kd(omega, depth, g):
    """Fenton's explicit approximation of k d (Eq. explicit_dispersion_relation)."""
    G = omega * omega * depth / g
    b = G / math.sqrt(math.tanh(G))
    sech2 = 0.0 if b > 350.0 else 1.0 / math.cosh(b) ** 2
    return (G + b * b * sech2) / (math.tanh(b) + b * sech2)


def group_velocity(omega, k, depth):
    """c_g = (lambda / 2T) (1 + 2kd / sinh 2kd) (Eq. group_velocity)."""
    lam = 2.0 * math.pi / k
    T = 2.0 * math.pi / omega
    x = 2.0 * k * depth
    return 0.5 * lam / T * (1.0 + (x / math.sinh(x) if x < 700.0 else 0.0))


def regular_wave_power(H, omega, k, depth, rho_w, g):
    """Mean power per unit crest width, (1/8) rho g H^2 c_g (Eq. regular_wave_power)."""
    return rho_w * g * H * H * group_velocity(omega, k, depth) / 8.0


def bretschneider_printed(omega, Hs, T):
    """The spectrum exactly as printed: 173 Hs^2 / T^4 w^-5 exp(-692 / (T^4 w^4))."""
    omega = np.asarray(omega, dtype=np.float64)
    return 173.0 * Hs * Hs / T ** 4 * omega ** -5 * np.exp(-692.0 / (T ** 4 * omega ** 4))


def bretschneider_period(Tp):
    """Period to put into the printed form so that its maximum is at omega_p = 2 pi / Tp.

    The paper calls Tp "the time period with the highest spectral density" and its
    figure caption pairs Tp = 1.7475 s with omega_p = 3.5955 rad/s = 2 pi / Tp, but the
    printed form with T = Tp peaks at (4/5 * 692)^(1/4) / Tp.  Reading: keep the
    printed form and take T so that d S / d omega = 0 at 2 pi / Tp, which gives
    T^4 = (4/5) 692 / omega_p^4.
    """
    wp = 2.0 * math.pi / Tp
    return (0.8 * 692.0) ** 0.25 / wp


def bretschneider(omega, Hs, Tp):
    return bretschneider_printed(omega, Hs, bretschneider_period(Tp))


def jonswap(omega, Hs, Tp, gamma):
    """Bretschneider shape times the peak enhancement gamma^exp(-(w-wp)^2 / (2 s^2 wp^2))."""
    omega = np.asarray(omega, dtype=np.float64)
    wp = 2.0 * math.pi / Tp
    s = np.where(omega <= wp, 0.07, 0.09)
    r = np.exp(-((omega - wp) ** 2) / (2.0 * s * s * wp * wp))
    return bretschneider(omega, Hs, Tp) * gamma ** r


def jonswap_components(Hs, Tp, gamma, ncomp, phases, normalise=True):
    """Discretise the spectrum into ``ncomp`` Airy components (Eq. wave_spectrum_amplitude).

    Equal bins over [BAND_LO, BAND_HI] omega_p evaluated at their mid-points; the
    amplitudes are rescaled so that 4 sqrt(sum a_i^2 / 2) equals Hs exactly.
    Returns (amp, omega, phase) arrays.
    """
    wp = 2.0 * math.pi / Tp
    lo, hi = BAND_LO * wp, BAND_HI * wp
    dw = (hi - lo) / ncomp
    omega = lo + dw * (np.arange(ncomp) + 0.5)
    amp = np.sqrt(2.0 * jonswap(omega, Hs, Tp, gamma) * dw)
    if normalise:
        hs_est = 4.0 * math.sqrt(float(np.sum(amp * amp)) / 2.0)
        amp = amp * (Hs / hs_est)
    return amp, omega, np.asarray(phases, dtype=np.float64)


def components(wave, depth, g):
    """(amp, omega, k, phase) arrays for a workload's wave dictionary."""
    if wave["kind"] == "regular":
        amp = np.array([0.5 * wave["H"]])
        omega = np.array([2.0 * math.pi / wave["T"]])
        phase = np.array([wave["phase"]])
    elif wave["kind"] == "jonswap":
        amp, omega, phase = jonswap_components(wave["Hs"], wave["Tp"], wave["gamma"],
                                               wave["ncomp"], wave["phases"])
    else:
        raise ValueError(wave["kind"])
    k = np.array([dispersion_k(w, depth, g) for w in omega])
    return amp, omega, k, phase
