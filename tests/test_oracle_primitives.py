"""Pins of the oracle's primitives: Philox4x32-10 against its published
known answers, the u32 -> [0,1) map, the Student t CDF / quantile against
scipy and closed forms, and the two-pass mean / variance."""
import math
import os

import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(O.philox4x32_10(ctr, key)) == out


def test_philox_counter_sensitivity():
    # every counter word and key word changes every output word (avalanche)
    base = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert np.all(O.philox4x32_10(c, [5, 6]) != base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert np.all(O.philox4x32_10([1, 2, 3, 4], k) != base)


def test_u01_exact_and_in_range():
    assert O.u01(0) == 0.0
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert O.u01(0x000000FF) == 0.0          # low 8 bits discarded
    assert O.u01(0x00000100) == 2.0 ** -24
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64):
        u = O.u01(int(x))
        assert 0.0 <= u < 1.0
        assert np.float32(u) == u            # exactly representable in FP32


@pytest.mark.parametrize("nu", [1, 2, 3, 7, 15, 63, 255, 511])
def test_t_cdf_matches_scipy(nu):
    for t in np.linspace(-8, 8, 41):
        assert O.t_cdf(t, nu) == pytest.approx(st.t.cdf(t, nu), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("nu", [1023, 4095, 8191])
def test_t_cdf_large_dof(nu):
    # lgamma(a+b) - lgamma(a) - lgamma(b) cancels ~1e-12 relative at a ~ 4e3
    for t in [-4.0, -2.0, -1.645, -0.5, 0.0, 0.7, 3.0]:
        assert O.t_cdf(t, nu) == pytest.approx(st.t.cdf(t, nu), rel=1e-9, abs=1e-15)


def test_t_cdf_closed_forms():
    for t in np.linspace(-20, 20, 81):
        # nu = 1 is the Cauchy distribution
        assert O.t_cdf(t, 1) == pytest.approx(0.5 + math.atan(t) / math.pi, abs=1e-14)
        # nu = 2 has F(t) = 1/2 + t / (2 sqrt(2 + t^2))
        assert O.t_cdf(t, 2) == pytest.approx(0.5 + t / (2 * math.sqrt(2 + t * t)), abs=1e-14)
    # normal limit
    for t in [-2.5, -1.0, 0.3]:
        assert O.t_cdf(t, 1e7) == pytest.approx(st.norm.cdf(t), abs=1e-7)
    assert O.t_cdf(0.0, 17) == pytest.approx(0.5, abs=1e-15)
    assert O.t_cdf(-math.inf, 5) == 0.0 and O.t_cdf(math.inf, 5) == 1.0


def test_betainc_matches_scipy():
    rng = np.random.default_rng(2)
    for _ in range(200):
        a, b = rng.uniform(0.2, 50, size=2)
        x = rng.uniform(0, 1)
        assert O.betainc(a, b, x) == pytest.approx(sp.betainc(a, b, x), rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("nu", [15, 255, 4095])
@pytest.mark.parametrize("p", [0.01, 0.025, 0.05, 0.95])
def test_t_ppf_inverts_cdf(nu, p):
    t = O.t_ppf(p, nu)
    assert t == pytest.approx(st.t.ppf(p, nu), rel=1e-9)
    assert O.t_cdf(t, nu) == pytest.approx(p, rel=1e-12)


def test_mean_var_two_pass():
    rng = np.random.default_rng(3)
    for n in [2, 3, 16, 257, 8192]:
        y = rng.normal(5.0, 0.01, size=n)   # large mean, small spread: naive sums lose digits
        m, v = O.mean_var(y)
        assert m == pytest.approx(float(np.mean(y)), rel=1e-14)
        assert v == pytest.approx(float(np.var(y, ddof=1)), rel=1e-10)
    m, v = O.mean_var(np.full(100, 2.5))
    assert m == 2.5 and v == 0.0
