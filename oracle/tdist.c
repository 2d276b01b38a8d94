/* Student t distribution for the one-tailed test of Sec. 3.2 (Eq. 7).
 * Test infrastructure only.
 *
 * F_nu(t) = 1/2 I_x(nu/2, 1/2) for t < 0 and 1 - 1/2 I_x(nu/2, 1/2) for
 * t >= 0, with x = nu / (nu + t^2) and I the regularized incomplete beta
 * function.  I_x(a, b) = x^a (1-x)^b / (a B(a,b)) * K(a, b, x), where K is
 * the continued fraction 1/(1+ d1/(1+ d2/(1+ ...))) with
 *   d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1)),
 *   d_{2m}   =  m (b-m) x / ((a+2m-1)(a+2m)),
 * evaluated by the modified Lentz method; for x above (a+1)/(a+b+2) the
 * symmetry I_x(a,b) = 1 - I_{1-x}(b,a) keeps the fraction convergent. */
#include <math.h>

#include "oracle.h"

static double betacf(double a, double b, double x) {
    const double tiny = 1e-300, eps = 1e-16;
    double f = 1.0, c = 1.0, dd = 1.0 - (a + b) * x / (a + 1.0);
    if (fabs(dd) < tiny) dd = tiny;
    dd = 1.0 / dd;
    f = dd;
    for (int m = 1; m <= 100000; ++m) {
        /* even step d_{2m} */
        double num = m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
        dd = 1.0 + num * dd;
        if (fabs(dd) < tiny) dd = tiny;
        c = 1.0 + num / c;
        if (fabs(c) < tiny) c = tiny;
        dd = 1.0 / dd;
        f *= dd * c;
        /* odd step d_{2m+1} */
        num = -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
        dd = 1.0 + num * dd;
        if (fabs(dd) < tiny) dd = tiny;
        c = 1.0 + num / c;
        if (fabs(c) < tiny) c = tiny;
        dd = 1.0 / dd;
        double delta = dd * c;
        f *= delta;
        if (fabs(delta - 1.0) < eps) break;
    }
    return f;
}

double orc_betainc(double a, double b, double x) {
    if (x <= 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    double lbt = lgamma(a + b) - lgamma(a) - lgamma(b) + a * log(x) + b * log1p(-x);
    double bt = exp(lbt);
    if (x < (a + 1.0) / (a + b + 2.0)) return bt * betacf(a, b, x) / a;
    return 1.0 - bt * betacf(b, a, 1.0 - x) / b;
}

double orc_t_cdf(double t, double nu) {
    if (isnan(t)) return NAN;
    if (isinf(t)) return t > 0 ? 1.0 : 0.0;
    double x = nu / (nu + t * t);
    double tail = 0.5 * orc_betainc(0.5 * nu, 0.5, x);
    return t < 0.0 ? tail : 1.0 - tail;
}

double orc_t_ppf(double p, double nu) {
    if (!(p > 0.0 && p < 1.0)) return NAN;
    double lo = -1.0, hi = 1.0;
    while (orc_t_cdf(lo, nu) > p) lo *= 2.0;
    while (orc_t_cdf(hi, nu) < p) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (orc_t_cdf(mid, nu) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}
