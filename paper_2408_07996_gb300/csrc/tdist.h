// tdist.h -- Student t critical values for the test of Eq. 7 (host, FP64).
#pragma once

namespace mcev {

// P(T <= t) for Student's t with integer nu >= 1 degrees of freedom.
double t_cdf_int(double t, int nu);
// t with P(T <= t) = p (0 < p < 1), by bisection on t_cdf_int.
double t_quantile_int(double p, int nu);

}  // namespace mcev
