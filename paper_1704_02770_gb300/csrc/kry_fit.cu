// Power-law decay exponent of the survival observables (Sec. 4): C(t) ~ a t^-gamma.
//
// The exponent is the least-squares slope of log C against log t over the output times of a
// window [t_min, t_max] (gamma = -slope); it reads a few dozen host values produced by the
// evolution, so it is host arithmetic with no device work.
#include <cmath>

#include "kry_internal.cuh"

using namespace kry;

extern "C" int kry_decay_exponent(const double *t, const double *C, int n, double t_min, double t_max,
                                  double *gamma, double *log_a)
{
    if (!t || !C || !gamma || n < 2 || !(t_min > 0.0) || !(t_max >= t_min)) {
        set_error("kry_decay_exponent: bad arguments (need t, C, gamma, n >= 2, 0 < t_min <= t_max)");
        return KRY_EINVAL;
    }
    // two passes: the means, then the centred sums (no cancellation between large sums)
    int cnt = 0;
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(t[i] >= t_min && t[i] <= t_max)) continue;
        if (!(C[i] > 0.0) || !std::isfinite(C[i])) {
            set_error("kry_decay_exponent: C(t) must be positive inside the window (index %d)", i);
            return KRY_EINVAL;
        }
        mx += std::log(t[i]);
        my += std::log(C[i]);
        ++cnt;
    }
    if (cnt < 2) { set_error("kry_decay_exponent: fewer than two times inside the window"); return KRY_EINVAL; }
    mx /= cnt;
    my /= cnt;
    double sxx = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(t[i] >= t_min && t[i] <= t_max)) continue;
        const double dx = std::log(t[i]) - mx;
        sxx += dx * dx;
        sxy += dx * (std::log(C[i]) - my);
    }
    if (!(sxx > 0.0)) { set_error("kry_decay_exponent: the window holds a single distinct time"); return KRY_EINVAL; }
    const double slope = sxy / sxx;
    *gamma = -slope;
    if (log_a) *log_a = my - slope * mx;
    return KRY_OK;
}
