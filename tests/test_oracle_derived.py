"""Pins of the oracle's derived distributions (Table "continuous"; Sec. 3.1
"Gamma and related distributions", "Extreme value and Weibull
distributions"): each against its textbook law (SciPy's CDF), and against
identities that tie it to another oracle routine by a different path (a
special parameter value, or a relation between two laws on the same draws)."""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

N = 40_000
P_MIN = 1e-4


def _fill(orc, name, *params, seed=7, n=N, engine="xoshiro256pp"):
    return orc.fill_derived(orc.gen(engine, seed), name, n, *params)


@pytest.mark.parametrize("name,params,law", [
    ("unif", (-2.0, 3.0), stats.uniform(loc=-2.0, scale=5.0)),
    ("normal_ms", (1.5, 2.0), stats.norm(loc=1.5, scale=2.0)),
    ("lognormal", (0.3, 0.7), stats.lognorm(s=0.7, scale=math.exp(0.3))),
    ("exp_scale", (2.5,), stats.expon(scale=2.5)),
    ("gamma_scale", (2.5, 0.5), stats.gamma(a=2.5, scale=0.5)),
    ("gamma_scale", (0.4, 3.0), stats.gamma(a=0.4, scale=3.0)),
    ("chi2", (5.0,), stats.chi2(5.0)),
    ("chi2", (1.3,), stats.chi2(1.3)),
    ("gumbel", (1.0, 2.0), stats.gumbel_r(loc=1.0, scale=2.0)),
    ("pareto", (2.0, 3.0), stats.pareto(b=3.0, scale=2.0)),
    ("weibull", (1.7, 2.0), stats.weibull_min(c=1.7, scale=2.0)),
    ("gpd", (0.5, 1.5, 0.3), stats.genpareto(c=0.3, loc=0.5, scale=1.5)),
    ("gpd", (0.5, 1.5, -0.4), stats.genpareto(c=-0.4, loc=0.5, scale=1.5)),
    ("gpd", (-1.0, 2.0, 0.0), stats.genpareto(c=0.0, loc=-1.0, scale=2.0)),
    ("f", (5.0, 7.0), stats.f(5.0, 7.0)),
    ("f", (3.0, 3.0), stats.f(3.0, 3.0)),
    ("skew_normal", (1.0, 2.0, 4.0), stats.skewnorm(a=4.0, loc=1.0, scale=2.0)),
    ("skew_normal", (0.0, 1.0, -2.0), stats.skewnorm(a=-2.0)),
    ("t", (3.0,), stats.t(3.0)),
    ("t", (0.8,), stats.t(0.8)),
    ("t", (1.0,), stats.cauchy()),
], ids=lambda x: str(x) if not hasattr(x, "dist") else x.dist.name)
def test_derived_against_law(orc, name, params, law):
    x = _fill(orc, name, *params)
    assert stats.kstest(x, law.cdf).pvalue > P_MIN, (name, params)
    # the mean too, where it exists and the variance is finite
    m, v = law.stats(moments="mv")
    if np.isfinite(m) and np.isfinite(v) and v > 0:
        assert abs(x.mean() - m) < 6 * math.sqrt(v / N), (name, params, x.mean(), m)


def test_weibull_shape_one_is_scaled_exponential(orc):
    """pow(E, 1) is E, so Weibull(1, lambda) repeats Exp(lambda) bit for bit
    on the same stream (pow's exponent is 1/k, not k)."""
    a = _fill(orc, "weibull", 1.0, 2.5, seed=3)
    b = _fill(orc, "exp_scale", 2.5, seed=3)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_pareto_log_recovers_the_exponential(orc):
    """alpha log(X / x_m) = E for Pareto(x_m, alpha) = x_m exp(E / alpha)."""
    x = _fill(orc, "pareto", 2.0, 3.0, seed=5)
    e = orc.fill(orc.gen("xoshiro256pp", 5), "exp", N)
    assert np.allclose(3.0 * np.log(x / 2.0), e, rtol=1e-13, atol=1e-14)


def test_lognormal_log_recovers_the_normal(orc):
    x = _fill(orc, "lognormal", 0.3, 0.7, seed=9)
    z = _fill(orc, "normal_ms", 0.3, 0.7, seed=9)
    assert np.allclose(np.log(x), z, rtol=1e-14, atol=1e-15)


def test_gpd_is_continuous_in_xi_at_zero(orc):
    """The two branches of the generalized Pareto formula meet the shifted
    exponential as xi -> 0 from either side (same draws)."""
    z0 = _fill(orc, "gpd", 0.5, 1.5, 0.0, seed=11)
    for xi in (1e-7, -1e-7):
        z = _fill(orc, "gpd", 0.5, 1.5, xi, seed=11)
        e = (z0 - 0.5) / 1.5
        assert np.allclose(z, z0, rtol=0, atol=1.5 * (abs(xi) * (e * e).max() + 1e-8))


def test_f_is_the_beta_odds_ratio(orc):
    """F = (X/nu1)/(Y/nu2) and B = X/(X+Y) from the same draws, so
    F = (nu2/nu1) B/(1-B): X is drawn before Y in both."""
    f = _fill(orc, "f", 5.0, 7.0, seed=13)
    b = orc.fill(orc.gen("xoshiro256pp", 13), "beta", N, 2.5, 3.5)
    assert np.allclose(f, (7.0 / 5.0) * b / (1.0 - b), rtol=1e-12)


def test_chi2_is_twice_gamma_half_nu(orc):
    x = _fill(orc, "chi2", 3.0, seed=17)
    g = orc.fill(orc.gen("xoshiro256pp", 17), "gamma", N, 1.5)
    assert np.array_equal(x, 2.0 * g)


def test_skew_normal_zero_alpha_is_the_second_normal(orc):
    """alpha = 0 gives delta = 0: z is the second normal of each pair."""
    x = _fill(orc, "skew_normal", 0.0, 1.0, 0.0, seed=19, n=5000)
    z = orc.fill(orc.gen("xoshiro256pp", 19), "normal", 10_000)
    assert np.array_equal(x, z[1::2])


def test_gumbel_and_unif_ranges(orc):
    u = _fill(orc, "unif", -2.0, 3.0, seed=23)
    assert u.min() >= -2.0 and u.max() < 3.0
    g = _fill(orc, "gumbel", 0.0, 1.0, seed=23)
    w = orc.fill(orc.gen("xoshiro256pp", 23), "uniform", N)
    # F(x) = exp(-exp(-x)) recovers the uniform draw
    assert np.allclose(np.exp(-np.exp(-g)), w, rtol=1e-12, atol=1e-15)


def test_cr_pow_against_mpmath(orc):
    rng = np.random.default_rng(5)
    mp.mp.prec = 200
    xs = np.exp(rng.uniform(-30, 3, 300))
    ys = rng.uniform(0.05, 4.0, 300)
    for x, y in zip(xs, ys):
        ref = float(mp.power(mp.mpf(float(x)), mp.mpf(float(y))))
        assert orc.cr_pow(x, y) == ref, (x, y)


def test_bad_parameters_are_refused(orc):
    g = orc.gen("xoshiro256pp", 1)
    with pytest.raises(ValueError):
        orc.fill_derived(g, "chi2", 4, -1.0)
    with pytest.raises(ValueError):
        orc.fill_derived(g, "f", 4, 2.0, 0.0)


def test_t_draws_the_normal_first(orc):
    """With nu huge, V / nu -> 1 and t -> Z: the first output follows the
    first normal of the stream (Z is drawn before V)."""
    t = _fill(orc, "t", 1e10, seed=29, n=1)
    z = orc.fill(orc.gen("xoshiro256pp", 29), "normal", 1)
    assert abs(t[0] - z[0]) <= 1e-4 * abs(z[0])
    big = _fill(orc, "t", 1e8, seed=31)
    assert stats.kstest(big, "norm").pvalue > P_MIN
