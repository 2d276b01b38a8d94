"""Pins of the oracle's Alg. 1 detector (Sec. 3.2-3.3) on synthetic
log-luminance samples: the t statistic and its degrees of freedom against
scipy's textbook t-tests, the one-tailed direction and alpha calibration,
the sampling schedule, the event rule and the reference update."""
import numpy as np
import pytest
import scipy.stats as st

import oracle as O


def det(**kw):
    d = dict(C=0.2, alpha=0.05, spp_min=16, spp_batch=16, spp_max=256, variant=O.ONE_TAILED,
             se_mode=O.SE_PAPER)
    d.update(kw)
    return O.Detect(**d)


def test_t_value_is_one_sample_t_when_reference_is_exact():
    # With s_a^2 = 0 the t-value of Eq. 7 is the one-sample t statistic of the
    # gaps y - mu_a against the threshold C, with n_b - 1 degrees of freedom.
    rng = np.random.default_rng(10)
    d = det(spp_min=64, spp_batch=64, spp_max=512)
    for trial in range(50):
        mu_a = rng.normal()
        y = mu_a + 0.2 + rng.normal(0.05, 0.7, size=512)
        r = O.detect_pixel(d, y, (512, mu_a, 0.0))
        res = st.ttest_1samp(y[:64] - mu_a, popmean=0.2, alternative="less")
        tcrit = st.t.ppf(0.05, 63)
        # margin_t includes the first test, whose t is scipy's statistic
        first_margin = abs(res.statistic - tcrit)
        assert r["margin_t"] <= first_margin + 1e-9
        stop_first = res.pvalue < 0.05
        if stop_first:
            assert r["n"] == 64
            assert r["margin_t"] == pytest.approx(first_margin, rel=1e-9, abs=1e-9)
        else:
            assert r["n"] > 64


def test_t_value_uses_both_variances_over_n_b():
    # With n_a = n_b the paper's standard error sqrt((s_a^2 + s_b^2)/N) equals
    # Welch's sqrt(s_a^2/n_a + s_b^2/n_b); scipy's Welch statistic on
    # (y_b - C, y_a) is then the t-value of Eq. 7.
    rng = np.random.default_rng(11)
    n = 32
    d = det(spp_min=n, spp_batch=n, spp_max=4 * n)
    checked = 0
    for _ in range(40):
        ya = rng.normal(0.0, 0.3, size=n)
        yb = rng.normal(0.05, 0.3, size=4 * n)
        ma, va = float(np.mean(ya)), float(np.var(ya, ddof=1))
        if np.mean(yb[:n]) < ma:
            continue
        r = O.detect_pixel(d, yb, (n, ma, va))
        tw = st.ttest_ind(yb[:n] - 0.2, ya, equal_var=False).statistic
        tcrit = st.t.ppf(0.05, n - 1)
        if r["n"] == n:  # stopped at the first test: margin is that test's
            assert r["margin_t"] == pytest.approx(abs(tw - tcrit), rel=1e-9)
            assert tw < tcrit
            checked += 1
        else:
            assert tw >= tcrit
            assert r["margin_t"] <= abs(tw - tcrit) + 1e-9
    assert checked > 0


def test_one_tailed_first_look_rejects_at_rate_alpha():
    # True gap exactly C and an exact reference: under H0 the statistic is
    # Student-t, so a single look stops with probability alpha.  C is many
    # standard errors above zero so that |mu_b - mu_a| never folds.
    rng = np.random.default_rng(12)
    trials, stops = 4000, 0
    d = det(C=2.0, spp_min=32, spp_batch=32, spp_max=64)
    for _ in range(trials):
        y = 2.0 + rng.normal(size=64)
        stops += O.detect_pixel(d, y, (64, 0.0, 0.0))["n"] == 32
    lo, hi = st.binom.ppf([0.0005, 0.9995], trials, 0.05)
    assert lo <= stops <= hi


def test_large_gap_runs_to_cap_and_fires():
    rng = np.random.default_rng(13)
    d = det()
    for sign in (+1, -1):
        y = sign * 1.0 + rng.normal(0, 0.3, size=256)
        r = O.detect_pixel(d, y, (256, 0.0, 0.09))
        assert r["n"] == 256 and r["event"] == sign
        assert r["ref"][0] == 256 and r["ref"][1] == pytest.approx(r["mean"])
        assert r["ref"][2] == pytest.approx(r["var"])


def test_no_event_keeps_reference():
    rng = np.random.default_rng(14)
    y = rng.normal(0, 0.1, size=256)
    r = O.detect_pixel(det(), y, (256, 0.01, 0.01))
    assert r["event"] == 0
    assert r["ref"] == (256, 0.01, 0.01)
    assert r["n"] == 16                      # decided at the first test


def test_schedule_and_early_stop_never_fires():
    rng = np.random.default_rng(15)
    d = det(spp_min=48, spp_batch=20, spp_max=300)
    allowed = {48 + 20 * k for k in range(13)} | {300}
    for _ in range(500):
        gap = rng.uniform(0, 0.4)
        y = gap + rng.normal(0, rng.uniform(0.05, 2.0), size=300)
        r = O.detect_pixel(d, y, (300, 0.0, rng.uniform(0, 0.5)))
        assert r["n"] in allowed
        if r["n"] < 300:
            assert r["event"] == 0          # a stop needs t < 0, i.e. gap < C
        if r["event"] != 0:
            assert r["n"] == 300


def test_event_rule_is_strict_and_signed():
    # values exactly representable in binary so the mean is exact
    d = det(C=0.25, spp_min=16, spp_batch=16, spp_max=16)
    for mu_b, expect in [(0.25, 0), (0.375, 1), (-0.375, -1), (-0.25, 0), (0.0, 0)]:
        y = np.full(16, mu_b)
        r = O.detect_pixel(d, y, (16, 0.0, 0.0))
        assert r["event"] == expect, mu_b


def test_zero_standard_error():
    d = det(spp_min=16, spp_batch=16, spp_max=64)
    r = O.detect_pixel(d, np.full(64, 0.1), (64, 0.0, 0.0))
    assert r["n"] == 16 and r["event"] == 0         # |gap| < C: stop
    r = O.detect_pixel(d, np.full(64, 0.5), (64, 0.0, 0.0))
    assert r["n"] == 64 and r["event"] == 1         # |gap| > C: run to the cap


def test_uniform_variant_never_stops():
    rng = np.random.default_rng(16)
    d = det(variant=O.UNIFORM)
    r = O.detect_pixel(d, rng.normal(0, 0.01, size=256), (256, 0.0, 0.0))
    assert r["n"] == 256


def test_prefix_property_adaptive_vs_uniform():
    # adaptive samples are a prefix of the uniform pixel's samples
    rng = np.random.default_rng(17)
    y = 0.1 + rng.normal(0, 0.4, size=256)
    ra = O.detect_pixel(det(), y, (256, 0.0, 0.16))
    m, v = O.mean_var(y[:ra["n"]])
    assert ra["mean"] == m and ra["var"] == v


def test_two_tailed_and_mean_only():
    rng = np.random.default_rng(18)
    # a clear event: two-tailed stops early, one-tailed runs to the cap
    y = 1.0 + rng.normal(0, 0.3, size=256)
    r2 = O.detect_pixel(det(variant=O.TWO_TAILED), y, (256, 0.0, 0.09))
    r1 = O.detect_pixel(det(), y, (256, 0.0, 0.09))
    assert r2["n"] == 16 and r2["event"] == 1
    assert r1["n"] == 256 and r1["event"] == 1
    # mean-only stops as soon as the mean gap is below C
    y = 0.05 + rng.normal(0, 2.0, size=256)
    y[:16] -= np.mean(y[:16]) - 0.05
    rm = O.detect_pixel(det(variant=O.MEAN_ONLY), y, (256, 0.0, 4.0))
    assert rm["n"] == 16


def test_welch_standard_error_option():
    rng = np.random.default_rng(19)
    n_a = 4096
    d = det(se_mode=O.SE_WELCH, spp_min=64, spp_batch=64, spp_max=128)
    y = 0.2 + rng.normal(0, 1.0, size=128)
    r = O.detect_pixel(d, y, (n_a, 0.0, 1.0))
    m = float(np.mean(y[:64]))
    t = (abs(m) - 0.2) / np.sqrt(1.0 / n_a + np.var(y[:64], ddof=1) / 64)
    assert r["margin_t"] <= abs(t - st.t.ppf(0.05, 63)) + 1e-9
