// tdist.cpp -- Student t distribution for integer degrees of freedom by the
// finite trigonometric series of Abramowitz & Stegun 26.7.3-26.7.4:
// with theta = atan(t / sqrt(nu)) and A(t|nu) = P(|T| <= t),
//   nu odd : A = (2/pi) (theta + sin(theta) (cos(theta) + 2/3 cos^3 + ...
//                 + (2*4*..*(nu-3)) / (1*3*..*(nu-2)) cos^(nu-2)))   (nu > 1)
//            A = 2 theta / pi                                         (nu = 1)
//   nu even: A = sin(theta) (1 + 1/2 cos^2 + 1*3/(2*4) cos^4 + ...
//                 + (1*3*..*(nu-3)) / (2*4*..*(nu-2)) cos^(nu-2))
// All terms are positive, so the sum is stable in FP64 for the nu <= 2^16
// the renderer needs.  The critical value of the one-tailed test (Sec. 3.2)
// is the alpha-quantile, found by bisection.
#include "tdist.h"

#include <cmath>

namespace mcev {

static double abs_prob(double t, int nu) {
    const double th = std::atan(std::fabs(t) / std::sqrt((double)nu));
    const double c = std::cos(th), s = std::sin(th), c2 = c * c;
    if (nu % 2 == 1) {
        if (nu == 1) return 2.0 * th / M_PI;
        double term = c, sum = c;
        for (int k = 1; 2 * k + 1 <= nu - 2; ++k) {
            term *= c2 * (2.0 * k) / (2.0 * k + 1.0);
            sum += term;
        }
        return 2.0 / M_PI * (th + s * sum);
    }
    double term = 1.0, sum = 1.0;
    for (int k = 1; 2 * k <= nu - 2; ++k) {
        term *= c2 * (2.0 * k - 1.0) / (2.0 * k);
        sum += term;
    }
    return s * sum;
}

double t_cdf_int(double t, int nu) {
    if (std::isnan(t)) return t;
    if (std::isinf(t)) return t > 0 ? 1.0 : 0.0;
    const double a = abs_prob(t, nu);
    return t >= 0.0 ? 0.5 * (1.0 + a) : 0.5 * (1.0 - a);
}

double t_quantile_int(double p, int nu) {
    if (!(p > 0.0 && p < 1.0)) return std::nan("");
    double lo = -1.0, hi = 1.0;
    while (t_cdf_int(lo, nu) > p) lo *= 2.0;
    while (t_cdf_int(hi, nu) < p) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (t_cdf_int(mid, nu) < p) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace mcev
