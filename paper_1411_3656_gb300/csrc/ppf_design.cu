// Host-side prototype filter design (Section 2): a truncated sinc shaped by a
// Hamming or Kaiser window, in FP64, rounded to FP32.
#include <cmath>
#include <cstdint>

#include "../../include/ppf.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Modified Bessel function of the first kind, order 0, by its power series
// I0(x) = sum_k ((x/2)^k / k!)^2; every term is positive, so the sum converges
// without cancellation.  Stops once a term no longer changes the sum.
double bessel_i0(double x)
{
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)k);
        const double next = sum + term;
        if (next == sum) break;
        sum = next;
    }
    return sum;
}

double sinc(double x)
{
    if (x == 0.0) return 1.0;
    const double a = kPi * x;
    return std::sin(a) / a;
}

}  // namespace

extern "C" ppf_status_t ppf_design_coeffs(int N, int T, ppf_window_t window, double beta, float* h_out)
{
    if (!h_out || N < 1 || T < 1) return PPF_ERR_INVALID_ARG;
    if (window != PPF_WINDOW_HAMMING && window != PPF_WINDOW_KAISER) return PPF_ERR_INVALID_ARG;
    if (window == PPF_WINDOW_KAISER && !(beta >= 0.0 && std::isfinite(beta))) return PPF_ERR_INVALID_ARG;
    const int64_t L = (int64_t)N * T;
    const double mid = 0.5 * (double)(L - 1);
    const double i0b = window == PPF_WINDOW_KAISER ? bessel_i0(beta) : 1.0;
    for (int64_t n = 0; n < L; ++n) {
        double w = 1.0;
        if (L > 1) {
            if (window == PPF_WINDOW_HAMMING) {
                w = 0.54 - 0.46 * std::cos(2.0 * kPi * (double)n / (double)(L - 1));
            } else {
                const double r = 2.0 * (double)n / (double)(L - 1) - 1.0;
                const double a = 1.0 - r * r;
                w = bessel_i0(beta * std::sqrt(a > 0.0 ? a : 0.0)) / i0b;
            }
        }
        h_out[n] = (float)(sinc(((double)n - mid) / (double)N) * w);
    }
    return PPF_OK;
}
