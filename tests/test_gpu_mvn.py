"""Multivariate normal x = mu + L z on the FP64 tensor cores against the
oracle's compensated (Dot2) product: Z bit-equal to the oracle's normal
stream (tails within 2 ulp), |x - x_oracle| <= 1e-13 (|mu| + |L| |z|)
componentwise; gradients dL/dmu = sum_j G_j and dL/dL = tril(G^T Z) within
1e-12 of the sum of magnitudes.  Shapes span one and several 64 x 64 tiles,
ragged d and n, and the workload sizes d = 64, 512 with n = 2^20
(sampled)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2605_05099_gb300 as rp
from paper_2605_05099_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(d, n, seed=3, stream=1, engine="xoshiro256pp"):
    mu_h, L_h = inputs.mvn_inputs(d)
    mu = torch.tensor(mu_h, device="cuda")
    L = torch.tensor(L_h, device="cuda")
    Z = torch.empty((n, d), dtype=torch.float64, device="cuda")
    X = torch.empty((n, d), dtype=torch.float64, device="cuda")
    pos = rp.rp_mvn(engine, seed, stream, 0, mu, L, Z, X)
    return mu_h, L_h, Z.cpu().numpy(), X.cpu().numpy(), pos


def _check_x(mu, L, Zh, Xh, rows=None):
    rows = np.arange(Zh.shape[0]) if rows is None else rows
    ref = oracle.mvn_apply(mu, L, Zh[rows])
    bound = 1e-13 * (np.abs(mu)[None, :] + np.abs(Zh[rows]) @ np.abs(L).T)
    err = np.abs(Xh[rows] - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("d,n", [(1, 1), (5, 37), (64, 1000), (100, 257), (130, 4101)])
def test_mvn_forward_matches_oracle(d, n):
    mu, L, Zh, Xh, pos = _run(d, n)
    g = oracle.gen("xoshiro256pp", 3, 1)
    zref = oracle.fill(g, "normal", n * d)
    assert pos == int(g.pos)
    zg, zo = Zh.ravel(), zref
    bad = np.nonzero(zg.view(np.int64) != zo.view(np.int64))[0]
    # only ziggurat tail outputs (|z| > R, values through a libm log) may differ, by 2 ulp
    R = oracle.zig_table(0)[3]
    assert np.all(np.abs(zo[bad]) > R), bad[:8]
    assert np.all(np.abs(zg.view(np.int64)[bad] - zo.view(np.int64)[bad]) <= 2)
    _check_x(mu, L, Zh, Xh)


@pytest.mark.parametrize("d,n", [(1, 3), (7, 100), (64, 3000), (130, 777)])
def test_mvn_grads_match_oracle(d, n):
    rng = np.random.default_rng(5)
    Zh = rng.standard_normal((n, d))
    Gh = rng.standard_normal((n, d))
    Z = torch.tensor(Zh, device="cuda")
    G = torch.tensor(Gh, device="cuda")
    gmu = torch.empty(d, dtype=torch.float64, device="cuda")
    gL = torch.empty((d, d), dtype=torch.float64, device="cuda")
    rp.rp_mvn_grads(G, Z, gmu, gL)
    rmu, rL = oracle.mvn_grads(Gh, Zh)
    smu = np.abs(Gh).sum(0)
    sL = np.tril(np.abs(Gh).T @ np.abs(Zh))
    assert np.all(np.abs(gmu.cpu().numpy() - rmu) <= 1e-12 * smu + 1e-300)
    gLh = gL.cpu().numpy()
    assert np.all(np.triu(gLh, 1) == 0.0)
    assert np.all(np.abs(gLh - rL) <= 1e-12 * sL + 1e-300)


def test_mvn_autograd():
    d, n = 16, 2000
    mu_h, L_h = inputs.mvn_inputs(d)
    mu = torch.tensor(mu_h, device="cuda", requires_grad=True)
    L = torch.tensor(L_h, device="cuda", requires_grad=True)
    X = rp.MVN.apply(mu, L, n, "philox4x32_10", 3, 1, 0)
    G = torch.tensor(np.random.default_rng(2).standard_normal((n, d)), device="cuda")
    (X * G).sum().backward()
    g = oracle.gen("philox4x32_10", 3, 1)
    Zh = oracle.fill(g, "normal", n * d).reshape(n, d)
    rmu, rL = oracle.mvn_grads(G.cpu().numpy(), Zh)
    assert np.allclose(mu.grad.cpu().numpy(), rmu, rtol=0, atol=1e-9)
    assert np.allclose(L.grad.cpu().numpy(), rL, rtol=0, atol=1e-9)


@pytest.mark.parametrize("d", [64, 512])
def test_mvn_workload_size_sampled(d):
    """n = 2^20 samples: 256 sampled rows of X against Dot2, and sampled
    gradient entries against exact-rounded sums (math.fsum)."""
    n = 1 << 20
    mu_h, L_h = inputs.mvn_inputs(d)
    mu = torch.tensor(mu_h, device="cuda")
    L = torch.tensor(L_h, device="cuda")
    Z = torch.empty((n, d), dtype=torch.float64, device="cuda")
    X = torch.empty((n, d), dtype=torch.float64, device="cuda")
    rp.rp_mvn("xoshiro256pp", 3, 1, 0, mu, L, Z, X)
    rows = np.random.default_rng(0).choice(n, 256, replace=False)
    rows_t = torch.tensor(rows, device="cuda")
    Zs = Z[rows_t].cpu().numpy()
    Xs = X[rows_t].cpu().numpy()
    _check_x(mu_h, L_h, Zs, Xs)
    G = torch.tensor(np.random.default_rng(3).standard_normal((n, d)), device="cuda")
    gmu = torch.empty(d, dtype=torch.float64, device="cuda")
    gL = torch.empty((d, d), dtype=torch.float64, device="cuda")
    rp.rp_mvn_grads(G, Z, gmu, gL)
    Gh, Zh = G.cpu().numpy(), Z.cpu().numpy()
    gmu_h, gL_h = gmu.cpu().numpy(), gL.cpu().numpy()
    rng = np.random.default_rng(1)
    for _ in range(6):
        i = int(rng.integers(0, d))
        k = int(rng.integers(0, i + 1))
        col_i, col_k = Gh[:, i], Zh[:, k]
        ex = math.fsum((col_i * col_k).tolist())
        mag = float(np.abs(col_i * col_k).sum())
        assert abs(gL_h[i, k] - ex) <= 1e-12 * mag
        ex_mu = math.fsum(col_i.tolist())
        assert abs(gmu_h[i] - ex_mu) <= 1e-12 * float(np.abs(col_i).sum())
    assert np.all(np.triu(gL_h, 1) == 0.0)
