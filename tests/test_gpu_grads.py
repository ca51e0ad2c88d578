"""GPU pathwise gradients against the oracle's quadrature gradients (which
are pinned to mpmath and SciPy finite differences in test_oracle_grads_mvn):
per-sample dz/dtheta within 1e-12 relative (1e-9 in the extreme tails), and
the reduced gradient through torch.autograd against the compensated oracle
sum."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2605_05099_gb300 as rp
from gpu_util import gpu_fill

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _tol(ref, z, lo_tail, hi_tail):
    t = np.full_like(ref, 1e-12)
    t[(z < lo_tail) | (z > hi_tail)] = 1e-9
    return t


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0, 2.5, 3.0, 7.5, 30.0, 150.0])
def test_gamma_dzda(alpha):
    z, _ = gpu_fill("gamma", "xoshiro256pp", 7, None, 0, 3000, (alpha,))
    # add grid points spanning both regimes and the extreme tails
    from scipy import special
    us = np.concatenate([[1e-12, 1e-8, 1e-4], np.linspace(0.01, 0.99, 60), [1 - 1e-4, 1 - 1e-9]])
    z = np.concatenate([z, special.gammaincinv(alpha, us)])
    z = z[z > 0]
    zt = torch.tensor(z, device="cuda")
    dz = torch.empty_like(zt)
    rp.rp_gamma_grad(zt, alpha, dzda=dz)
    got = dz.cpu().numpy()
    ref = np.array([oracle.gamma_dzda(v, alpha) for v in z])
    lo, hi = special.gammaincinv(alpha, 1e-6), special.gammaincinv(alpha, 1 - 1e-6)
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.all(rel <= _tol(ref, z, lo, hi)), (alpha, float(rel.max()), z[np.argmax(rel)])


def _gamma_grad(z, alpha, g=None):
    zt = torch.tensor(z, device="cuda")
    dz = torch.empty_like(zt)
    gt = None if g is None else torch.tensor(g, device="cuda")
    s = rp.rp_gamma_grad(zt, alpha, g=gt, dzda=dz)
    return dz.cpu().numpy(), s


@pytest.mark.parametrize("alpha", [2.5, 30.0, 1.0000001])
def test_gamma_dzda_branch_boundary_and_edges(alpha):
    """z at and next to alpha + 1 (where the series gives way to the
    continued fraction), z <= 0 and NaN (gradient 0), in windows of every
    ragged length around the 256-sample sort window and the 32-lane batch."""
    a1 = alpha + 1.0
    near = [np.nextafter(a1, 0.0), a1, np.nextafter(a1, 2 * a1), a1 * (1 - 1e-9), a1 * (1 + 1e-9)]
    rng = np.random.default_rng(5)
    for n in (1, 31, 33, 255, 257, 1000):
        z = rng.gamma(alpha, size=n)
        pos = rng.choice(n, size=min(n, 5), replace=False)
        z[pos] = near[:len(pos)]
        if n > 20:
            z[7], z[11], z[13] = 0.0, -1.5, np.nan
        got, _ = _gamma_grad(z, alpha)
        ref = np.array([oracle.gamma_dzda(v, alpha) if v > 0 else 0.0 for v in z])
        zero = ~(z > 0)
        assert np.all(got[zero] == 0.0), (n, got[zero])
        rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
        assert np.all(rel <= 1e-12), (alpha, n, float(rel.max()), z[~zero][np.argmax(rel)])


def test_gamma_grad_full_size_sampled():
    """The timed workload (n = 2^26 gamma(2.5) variates, xoshiro256++ seed 7,
    upstream g ~ N(0, 1)): sampled per-sample gradients against the oracle,
    the reduced sum against the per-sample values, and a second call bit for
    bit equal (the sums have a fixed order)."""
    from paper_2605_05099_gb300 import inputs
    n, alpha = 1 << 26, 2.5
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    rp.rp_fill_gamma("xoshiro256pp", 7, rp.NO_STREAM, 0, alpha, z)
    g = torch.tensor(inputs.upstream_grads(n), device="cuda")
    dz = torch.empty_like(z)
    s1 = rp.rp_gamma_grad(z, alpha, g=g, dzda=dz)
    s2 = rp.rp_gamma_grad(z, alpha, g=g)
    assert s1 == s2
    idx = np.random.default_rng(9).choice(n, size=600, replace=False)
    it = torch.tensor(idx, device="cuda")
    zs, ds = z[it].cpu().numpy(), dz[it].cpu().numpy()
    ref = np.array([oracle.gamma_dzda(v, alpha) for v in zs])
    assert np.all(np.abs(ds - ref) <= 1e-12 * np.abs(ref))
    # NumPy's pairwise sum is within about log2(n) 2^-53 sum|x| of the exact sum
    prod = (g * dz).cpu().numpy()
    assert abs(s1 - float(prod.sum())) <= 1e-12 * float(np.abs(prod).sum())


@pytest.mark.parametrize("ab", [(0.5, 0.5), (2.0, 5.0), (0.7, 3.0), (3.0, 2.0), (30.0, 40.0)])
def test_beta_dzdab(ab):
    a, b = ab
    from scipy import special
    z, _ = gpu_fill("beta", "xoshiro256pp", 7, None, 0, 2000, ab)
    us = np.concatenate([[1e-10, 1e-6], np.linspace(0.01, 0.99, 60), [1 - 1e-6]])
    z = np.concatenate([z, special.betaincinv(a, b, us)])
    z = z[(z > 0) & (z < 1)]
    zt = torch.tensor(z, device="cuda")
    da, db = torch.empty_like(zt), torch.empty_like(zt)
    rp.rp_beta_grad(zt, a, b, dzda=da, dzdb=db)
    ref = np.array([oracle.beta_dzdab(v, a, b) for v in z])
    lo, hi = special.betaincinv(a, b, 1e-5), special.betaincinv(a, b, 1 - 1e-5)
    for got, r in ((da.cpu().numpy(), ref[:, 0]), (db.cpu().numpy(), ref[:, 1])):
        rel = np.abs(got - r) / np.abs(r)
        assert np.all(rel <= _tol(r, z, lo, hi)), (ab, float(rel.max()), z[np.argmax(rel)])


def test_beta_dzdab_split_and_edges():
    """z at and next to the split (a+1)/(a+b+2) between the two orientations,
    z outside (0, 1) and NaN (gradients 0), in ragged windows."""
    a, b = 2.0, 5.0
    sp = (a + 1) / (a + b + 2)
    near = [np.nextafter(sp, 0.0), sp, np.nextafter(sp, 1.0)]
    rng = np.random.default_rng(6)
    for n in (1, 33, 257, 700):
        z = rng.beta(a, b, size=n)
        pos = rng.choice(n, size=min(n, 3), replace=False)
        z[pos] = near[:len(pos)]
        if n > 20:
            z[5], z[9], z[12], z[15] = 0.0, 1.0, -0.5, np.nan
        zt = torch.tensor(z, device="cuda")
        da, db = torch.empty_like(zt), torch.empty_like(zt)
        rp.rp_beta_grad(zt, a, b, dzda=da, dzdb=db)
        ok = (z > 0) & (z < 1)
        ref = np.array([oracle.beta_dzdab(v, a, b) if 0 < v < 1 else (0.0, 0.0) for v in z])
        for got, r in ((da.cpu().numpy(), ref[:, 0]), (db.cpu().numpy(), ref[:, 1])):
            assert np.all(got[~ok] == 0.0)
            rel = np.abs(got[ok] - r[ok]) / np.abs(r[ok])
            assert np.all(rel <= 1e-12), (n, float(rel.max()), z[ok][np.argmax(rel)])


def test_autograd_gamma_and_beta():
    n = 1 << 14
    g = torch.tensor(np.random.default_rng(1).standard_normal(n), device="cuda")
    alpha = torch.tensor(2.5, dtype=torch.float64, requires_grad=True)
    z = rp.Gamma.apply(alpha, n, "xoshiro256pp", 7, rp.NO_STREAM, 0)
    (z * g).sum().backward()
    zn, gn = z.detach().cpu().numpy(), g.cpu().numpy()
    ref = math.fsum(gi * oracle.gamma_dzda(zi, 2.5) for gi, zi in zip(gn, zn))
    scale = math.fsum(abs(gi * oracle.gamma_dzda(zi, 2.5)) for gi, zi in zip(gn, zn))
    assert abs(alpha.grad.item() - ref) <= 1e-12 * scale
    a = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)
    z = rp.Beta.apply(a, b, n, "philox4x32_10", 3, rp.NO_STREAM, 0)
    (z * g).sum().backward()
    zn = z.detach().cpu().numpy()
    refs = [oracle.beta_dzdab(zi, 2.0, 5.0) for zi in zn]
    for got, k in ((a.grad.item(), 0), (b.grad.item(), 1)):
        ref = math.fsum(gi * r[k] for gi, r in zip(gn, refs))
        scale = math.fsum(abs(gi * r[k]) for gi, r in zip(gn, refs))
        assert abs(got - ref) <= 1e-12 * scale


def test_grad_argument_errors():
    L = rp.lib()
    import ctypes
    assert L.rp_gamma_grad(None, 1.0, None, 5, None, None, None) == -1
    assert L.rp_gamma_grad(ctypes.c_void_p(0x1000), -1.0, None, 5, ctypes.c_void_p(0x1000), None, None) == -2
    assert L.rp_beta_grad(ctypes.c_void_p(0x1000), 1.0, 0.0, None, 5, ctypes.c_void_p(0x1000), None, None, None, None) == -2


@pytest.mark.parametrize("ab", [(2.0, 5.0), (0.5, 0.5), (30.0, 31.0), (0.7, 3.0)])
def test_beta_xy_fill_keeps_the_gamma_pairs(ab):
    """rp_fill_beta_xy: the same z as rp_fill_beta bit for bit, and X, Y equal
    to the oracle's gamma pairs (X ~ Gamma(a) drawn before Y ~ Gamma(b))."""
    a, b = ab
    n = 50_003
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    x, y = torch.empty_like(z), torch.empty_like(z)
    p = rp.rp_fill_beta_xy("philox4x32_10", 9, rp.NO_STREAM, 11, a, b, z, x, y)
    ref = torch.empty_like(z)
    p2 = rp.rp_fill_beta("philox4x32_10", 9, rp.NO_STREAM, 11, a, b, ref)
    assert p == p2
    assert torch.equal(z.view(torch.int64), ref.view(torch.int64))
    xy = oracle.beta_pairs(oracle.gen("philox4x32_10", 9, None, pos=11), n, a, b)
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    tol = 0 if min(ab) >= 1 else 2   # the boost's libm exp on both gammas
    for got, ref_ in ((xs, xy[:, 0]), (ys, xy[:, 1])):
        d = np.abs(got.view(np.int64) - ref_.view(np.int64))
        assert int(d.max()) <= tol, (ab, int(d.max()))


@pytest.mark.parametrize("ab", [(2.0, 5.0), (0.5, 0.5), (30.0, 31.0)])
def test_beta_grad_composed(ab):
    """dz/da = Y/(X+Y)^2 dX/da and dz/db = -X/(X+Y)^2 dY/db on the fill's
    gamma pairs, per sample within 1e-12 of the oracle's composition of its
    quadrature gradients (1e-9 where a gamma lies in its extreme tails), and
    the sums with g within 1e-12 of sum |g dz|."""
    a, b = ab
    from scipy import special
    n = 4000
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    x, y = torch.empty_like(z), torch.empty_like(z)
    rp.rp_fill_beta_xy("xoshiro256pp", 3, rp.NO_STREAM, 0, a, b, z, x, y)
    g = torch.tensor(np.random.default_rng(2).standard_normal(n), device="cuda")
    da, db = torch.empty_like(z), torch.empty_like(z)
    sa, sb = rp.rp_beta_grad_composed(x, y, a, b, g=g, dzda=da, dzdb=db)
    xs, ys, gs = x.cpu().numpy(), y.cpu().numpy(), g.cpu().numpy()
    ref = np.array([oracle.beta_dzdab_composed(xi, yi, a, b) for xi, yi in zip(xs, ys)])
    tails = ((xs < special.gammaincinv(a, 1e-6)) | (xs > special.gammaincinv(a, 1 - 1e-6)) |
             (ys < special.gammaincinv(b, 1e-6)) | (ys > special.gammaincinv(b, 1 - 1e-6)))
    tol = np.where(tails, 1e-9, 1e-12)
    for got, r, s in ((da.cpu().numpy(), ref[:, 0], sa), (db.cpu().numpy(), ref[:, 1], sb)):
        assert np.all(np.abs(got - r) <= tol * np.abs(r)), (ab, float((np.abs(got - r) / np.abs(r)).max()))
        assert abs(s - math.fsum(gs * r)) <= 1e-12 * math.fsum(np.abs(gs * r))
    # sums only (no per-sample outputs) give the same values
    assert rp.rp_beta_grad_composed(x, y, a, b, g=g) == (sa, sb)
