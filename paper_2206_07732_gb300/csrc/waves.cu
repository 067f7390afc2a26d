// Host wave utilities of libwec (no device work).
//   wave_number ............ Eq. dispersion_relation, omega^2 = g k tanh(k d), by
//                            Newton iteration started from Fenton's explicit k d
//                            (Eq. explicit_dispersion_relation)
//   jonswap ................ Eq. wave_spectrum_amplitude over the Bretschneider shape
//                            (Eq. Bretshneider_wave_spec) times the JONSWAP peak factor
#include <cmath>

#include "internal.cuh"

namespace wec {

double wave_number_fenton_kd(double omega, double depth, double g)
{
    double G = omega * omega * depth / g;
    double b = G / std::sqrt(std::tanh(G));
    double sech2 = b > 350.0 ? 0.0 : 1.0 / (std::cosh(b) * std::cosh(b));
    return (G + b * b * sech2) / (std::tanh(b) + b * sech2);
}

double wave_number(double omega, double depth, double g)
{
    if (!(omega > 0.0)) return 0.0;
    double k = wave_number_fenton_kd(omega, depth, g) / depth;
    const double target = omega * omega / g;
    for (int it = 0; it < 60; ++it) {
        double kd = k * depth;
        double th = std::tanh(kd);
        double F = k * th - target;
        double dF = th + kd * (1.0 - th * th);
        double step = F / dF;
        k -= step;
        if (std::fabs(step) <= 2e-16 * k) break;
    }
    return k;
}

int jonswap(double Hs, double Tp, double gamma, int ncomp, double *amp, double *omega)
{
    const double wp = 2.0 * kPi / Tp;
    // Bretschneider constants as printed (173, 692); its period T is chosen so that
    // the maximum sits at wp: d/dw [w^-5 exp(-692 / (T^4 w^4))] = 0 -> T^4 = 0.8 * 692 / wp^4.
    const double T4 = 0.8 * 692.0 / (wp * wp * wp * wp);
    const double lo = (1.6 / 3.5955) * wp, hi = (20.0 / 3.5955) * wp;
    const double dw = (hi - lo) / ncomp;
    double e2 = 0.0;
    for (int c = 0; c < ncomp; ++c) {
        double w = lo + dw * (c + 0.5);
        double w4 = w * w * w * w;
        double sb = 173.0 * Hs * Hs / T4 / (w4 * w) * std::exp(-692.0 / (T4 * w4));
        double s = w <= wp ? 0.07 : 0.09;
        double r = std::exp(-(w - wp) * (w - wp) / (2.0 * s * s * wp * wp));
        double S = sb * std::pow(gamma, r);
        omega[c] = w;
        amp[c] = std::sqrt(2.0 * S * dw);
        e2 += amp[c] * amp[c];
    }
    double scale = e2 > 0.0 ? Hs / (4.0 * std::sqrt(0.5 * e2)) : 0.0;
    for (int c = 0; c < ncomp; ++c) amp[c] *= scale;
    return WEC_OK;
}

}  // namespace wec
