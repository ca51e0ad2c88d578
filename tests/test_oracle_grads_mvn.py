"""Pins of the oracle's pathwise gradients and MVN transform.

Gradients: dz/dtheta = -(dF/dtheta)(z)/f(z) for z = F^{-1}(u; theta).
Pinned against (i) mpmath: high-precision numerical derivative of the
regularised incomplete gamma / beta functions, (ii) central finite
differences of SciPy's quantile functions at fixed u, and (iii) the alpha = 1
closed form -(dP/dalpha)/f = ln z + gamma_E + e^z E1(z) (evaluated in mpmath).
MVN: Dot2 result against exact rational arithmetic (Fractions)."""
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest
from scipy import special

U_GRID = [1e-9, 1e-4, 0.01, 0.2, 0.5, 0.8, 0.99, 1 - 1e-6]


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0, 2.5, 3.0, 7.5, 30.0, 150.0])
def test_gamma_dzda_vs_mpmath(orc, alpha):
    mp.mp.dps = 40
    for u in U_GRID:
        z = float(special.gammaincinv(alpha, u))
        zz = mp.mpf(z)
        dP = mp.diff(lambda a: mp.gammainc(a, 0, zz, regularized=True), mp.mpf(alpha))
        f = zz ** (alpha - 1) * mp.exp(-zz) / mp.gamma(alpha)
        ref = float(-dP / f)
        got = orc.gamma_dzda(z, alpha)
        assert abs(got - ref) <= 1e-13 * abs(ref), (alpha, u, got, ref)


@pytest.mark.parametrize("alpha", [0.3, 2.5, 30.0])
def test_gamma_dzda_vs_quantile_fd(orc, alpha):
    for u in [0.01, 0.2, 0.5, 0.8, 0.99]:
        z = special.gammaincinv(alpha, u)
        h = 1e-5 * alpha
        fd = (special.gammaincinv(alpha + h, u) - special.gammaincinv(alpha - h, u)) / (2 * h)
        assert abs(orc.gamma_dzda(z, alpha) - fd) <= 1e-6 * abs(fd)


def test_gamma_dzda_alpha1_closed_form(orc):
    mp.mp.dps = 40
    for z in [1e-12, 1e-3, 0.1, 1.0, 5.0, 30.0, 200.0]:
        zz = mp.mpf(z)
        ref = float(mp.log(zz) + mp.euler + mp.exp(zz) * mp.e1(zz))
        assert abs(orc.gamma_dzda(z, 1.0) - ref) <= 1e-13 * abs(ref), z


@pytest.mark.parametrize("ab", [(0.5, 0.5), (2.0, 5.0), (0.7, 3.0), (3.0, 2.0), (30.0, 40.0)])
def test_beta_dzdab_vs_mpmath(orc, ab):
    a, b = ab
    mp.mp.dps = 40
    for u in U_GRID:
        z = float(special.betaincinv(a, b, u))
        if not 0 < z < 1:
            continue
        zz = mp.mpf(z)
        I = lambda aa, bb: mp.betainc(aa, bb, 0, zz, regularized=True)
        f = zz ** (a - 1) * (1 - zz) ** (b - 1) / mp.beta(a, b)
        ra = float(-mp.diff(lambda aa: I(aa, mp.mpf(b)), mp.mpf(a)) / f)
        rb = float(-mp.diff(lambda bb: I(mp.mpf(a), bb), mp.mpf(b)) / f)
        ga, gb = orc.beta_dzdab(z, a, b)
        assert abs(ga - ra) <= 1e-12 * abs(ra), (ab, u, ga, ra)
        assert abs(gb - rb) <= 1e-12 * abs(rb), (ab, u, gb, rb)


def test_beta_arcsine_symmetry(orc):
    """Beta(1/2,1/2) is the arcsine law; by the a<->b, z<->1-z symmetry
    dz/da(z) = -dz/db(1-z)."""
    for z in [0.01, 0.3, 0.5, 0.77]:
        ga, gb = orc.beta_dzdab(z, 0.5, 0.5)
        ga2, gb2 = orc.beta_dzdab(1 - z, 0.5, 0.5)
        assert abs(ga + gb2) <= 1e-12 * abs(ga)
        assert abs(gb + ga2) <= 1e-12 * abs(gb)


def test_digamma(orc):
    for x in [0.1, 0.3, 0.5, 1.0, 2.5, 7.3, 30.0, 1e3]:
        # recurrence to x >= 12 accumulates up to ~12 roundings
        assert abs(orc.digamma(x) - float(mp.digamma(x))) <= 3e-15 * max(1.0, abs(float(mp.digamma(x))))


def test_mvn_dot2_exact(orc):
    """x_i = mu_i + sum_k L_ik z_k: Dot2 is within one rounding of the exact
    rational value (here checked: |x - exact| <= 2 ulp(exact))."""
    rng = np.random.default_rng(3)
    d, n = 9, 40
    mu = rng.standard_normal(d)
    L = np.tril(rng.standard_normal((d, d)))
    Z = rng.standard_normal((n, d))
    X = orc.mvn_apply(mu, L, Z)
    for j in range(n):
        for i in range(d):
            ex = Fraction(mu[i]) + sum(Fraction(L[i, k]) * Fraction(Z[j, k]) for k in range(i + 1))
            assert abs(Fraction(X[j, i]) - ex) <= 2 * Fraction(np.spacing(abs(float(ex))))


def test_mvn_grads_exact(orc):
    rng = np.random.default_rng(4)
    d, n = 5, 30
    G = rng.standard_normal((n, d))
    Z = rng.standard_normal((n, d))
    gmu, gL = orc.mvn_grads(G, Z)
    for i in range(d):
        ex = sum(Fraction(G[j, i]) for j in range(n))
        assert abs(Fraction(gmu[i]) - ex) <= 2 * Fraction(np.spacing(abs(float(ex))))
        for k in range(d):
            ex = sum(Fraction(G[j, i]) * Fraction(Z[j, k]) for j in range(n)) if k <= i else 0
            assert abs(Fraction(gL[i, k]) - ex) <= 2 * Fraction(np.spacing(abs(float(ex)) or 1e-300))


def test_substream_recipe(orc):
    """Sec. 2.3 parallel-simulation recipe: xoshiro substream s = base jumped
    s times by 2^128; Philox substream s = base with key s."""
    base = orc.state_words(orc.gen("xoshiro256pp", 99))
    s = base
    for k in range(1, 4):
        s = orc.xoshiro_jump(s, 2 ** 128, "matrix")
        assert orc.state_words(orc.substream("xoshiro256pp", 99, k)) == s
    p = orc.substream("philox4x32_10", 99, 17)
    q = orc.gen("philox4x32_10", 99)
    assert p.s[0] == q.s[0] and p.s[1] == q.s[1] and p.s[2] == 17


@pytest.mark.parametrize("ab", [(2.0, 5.0), (0.5, 0.5), (0.7, 3.0)])
def test_beta_gradient_through_the_gamma_pair_is_unbiased(orc, ab):
    """The composition estimator dz/da = Y/(X+Y)^2 dX/da, dz/db = -X/(X+Y)^2 dY/db
    on the beta fill's own gamma pairs: its mean is d/da E[z] = b/(a+b)^2 and
    d/db E[z] = -a/(a+b)^2, and E[2 z dz/da] is d/da E[z^2] with
    E[z^2] = a(a+1)/((a+b)(a+b+1)); the implicit beta-CDF estimator on the
    same z has the same means (both within 5 standard errors)."""
    a, b = ab
    n = 20_000
    xy = orc.beta_pairs(orc.gen("xoshiro256pp", 5), n, a, b)
    z = xy[:, 0] / (xy[:, 0] + xy[:, 1])
    zb = orc.fill(orc.gen("xoshiro256pp", 5), "beta", n, a, b)
    assert np.array_equal(z.view(np.uint64), zb.view(np.uint64))   # the pairs are the fill's draws
    d = np.array([orc.beta_dzdab_composed(x, y, a, b) for x, y in xy])
    se = d.std(axis=0) / np.sqrt(n)
    assert abs(d[:, 0].mean() - b / (a + b) ** 2) < 5 * se[0]
    assert abs(d[:, 1].mean() + a / (a + b) ** 2) < 5 * se[1]
    m2 = lambda aa: aa * (aa + 1) / ((aa + b) * (aa + b + 1))
    dm2 = float(mp.diff(m2, mp.mpf(a)))
    v = 2 * z * d[:, 0]
    assert abs(v.mean() - dm2) < 5 * v.std() / np.sqrt(n)
    imp = np.array([orc.beta_dzdab(zz, a, b) for zz in z])
    diff = d - imp
    assert np.all(np.abs(diff.mean(axis=0)) < 5 * diff.std(axis=0) / np.sqrt(n))
