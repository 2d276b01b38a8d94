/* Statistical event detection, Alg. 1 and Sec. 3.2-3.3.  Test infrastructure
 * only; the readings of the paper this follows are:
 *
 *  - samples come in a first batch of spp_min, then batches of spp_batch,
 *    capped at spp_max (Sec. 3.3: first test at 256, then +64, cap 4096);
 *  - after each batch that leaves n < spp_max, the mean and the unbiased
 *    variance of all n log-luminance samples are recomputed (calcMeanVar);
 *  - t = (|mu_b - mu_a| - C) / sqrt((s_a^2 + s_b^2) / n_b)  (Eq. 7, N = n_b);
 *    the Welch form sqrt(s_a^2/n_a + s_b^2/n_b) is the optional se_mode;
 *  - one-tailed test towards "gap below C": stop sampling iff
 *    F_{n_b - 1}(t) < alpha (Sec. 3.2), F the Student t CDF;
 *  - zero standard error: stop iff |mu_b - mu_a| < C;
 *  - after sampling stops (test or cap): an event of polarity
 *    sign(mu_b - mu_a) fires iff |mu_b - mu_a| > C, and then the reference
 *    (mu_a, s_a^2) becomes (mu_b, s_b^2)  (Alg. 1, Eq. 1); one event per
 *    pixel per frame.
 * Variants (the paper's ablations, Sec. 3.2 discussion): two-tailed stops
 * when either tail is below alpha/2; mean-only stops iff |mu_b - mu_a| < C;
 * uniform never stops before spp_max (the baseline of Sec. 4). */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

void orc_mean_var(const double* y, int64_t n, double* mean, double* var) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += y[i];
    double m = s / (double)n;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) q += (y[i] - m) * (y[i] - m);
    *mean = m;
    *var = n > 1 ? q / (double)(n - 1) : 0.0;
}

void orc_detect_pixel_cb(const orc_detect* d, orc_draw_fn draw, void* ctx,
                         int64_t* ref_n, double* ref_mean, double* ref_var,
                         int8_t* event, int32_t* n_used, double* mean, double* var,
                         double* margin_t, double* margin_c) {
    double* y = (double*)malloc(sizeof(double) * (d->spp_max > 0 ? d->spp_max : 1));
    int64_t n = 0;
    double mb = 0.0, vb = 0.0, mt = INFINITY;
    double t_lo = NAN, t_hi = NAN;
    while (n < d->spp_max) {
        int64_t nb = n == 0 ? d->spp_min : d->spp_batch;
        if (nb > d->spp_max - n) nb = d->spp_max - n;
        draw(ctx, n, nb, y + n);
        n += nb;
        orc_mean_var(y, n, &mb, &vb);
        if (n >= d->spp_max || d->variant == ORC_UNIFORM) continue;
        double gap = fabs(mb - *ref_mean);
        int stop;
        if (d->variant == ORC_MEAN_ONLY) {
            stop = gap < d->C;
        } else {
            double se2 = d->se_mode == ORC_SE_WELCH ? *ref_var / (double)*ref_n + vb / (double)n
                                                    : (*ref_var + vb) / (double)n;
            if (se2 == 0.0) {
                stop = gap < d->C;
            } else {
                double t = (gap - d->C) / sqrt(se2);
                double P = orc_t_cdf(t, (double)(n - 1));
                if (d->variant == ORC_TWO_TAILED) {
                    stop = P < 0.5 * d->alpha || P > 1.0 - 0.5 * d->alpha;
                    t_lo = orc_t_ppf(0.5 * d->alpha, (double)(n - 1));
                    t_hi = -t_lo;
                    double m1 = fmin(fabs(t - t_lo), fabs(t - t_hi));
                    if (m1 < mt) mt = m1;
                } else {
                    stop = P < d->alpha;
                    t_lo = orc_t_ppf(d->alpha, (double)(n - 1));
                    if (fabs(t - t_lo) < mt) mt = fabs(t - t_lo);
                }
            }
        }
        if (stop) break;
    }
    double delta = mb - *ref_mean;
    double gap = fabs(delta);
    int8_t ev = 0;
    if (gap > d->C) {
        ev = delta > 0.0 ? 1 : -1;
        *ref_n = n;
        *ref_mean = mb;
        *ref_var = vb;
    }
    *event = ev;
    *n_used = (int32_t)n;
    *mean = mb;
    *var = vb;
    *margin_t = mt;
    *margin_c = fabs(gap - d->C);
    free(y);
}

typedef struct {
    const double* y;
} array_src;

static void draw_array(void* ctx, int64_t k0, int64_t count, double* out) {
    const array_src* a = (const array_src*)ctx;
    for (int64_t k = 0; k < count; ++k) out[k] = a->y[k0 + k];
}

void orc_detect_pixel(const orc_detect* d, const double* y,
                      int64_t* ref_n, double* ref_mean, double* ref_var,
                      int8_t* event, int32_t* n_used, double* mean, double* var,
                      double* margin_t, double* margin_c) {
    array_src a = {y};
    orc_detect_pixel_cb(d, draw_array, &a, ref_n, ref_mean, ref_var, event, n_used, mean, var,
                        margin_t, margin_c);
}
