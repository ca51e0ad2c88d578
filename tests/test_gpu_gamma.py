"""GPU parity of the Marsaglia-Tsang gamma and the beta fills against the
oracle: identical consumed words; outputs bit-exact when no transcendental
enters the value (alpha >= 1 and beta with both shapes >= 1), and within a
few ulp when the alpha < 1 boost exp(log(U)/alpha) does (libm exp on the GPU,
correctly rounded exp in the oracle)."""
import numpy as np
import pytest
import torch

from gpu_util import BOOST_ULP, gpu_fill, oracle_fill

pytestmark = pytest.mark.gpu

ENGINES = ["xoshiro256pp", "pcg64dxsm", "philox4x32_10", "philox4x64_10", "xoshiro256ss"]
SIZES = [1, 7, 1000, 40_000, (1 << 17) + 3]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def max_ulp(a, b):
    """largest distance in ulps (integer arithmetic on the bit patterns of
    non-negative doubles)"""
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    return int(np.max(np.abs(ia - ib))) if len(ia) else 0


def check(dist, engine, seed, n, params, ulp, pos=0, stream=None):
    g, gpos = gpu_fill(dist, engine, seed, stream, pos, n, params)
    o, opos = oracle_fill(dist, engine, seed, stream, pos, n, params)
    assert gpos == opos, (dist, engine, params, n, gpos, opos)
    assert np.all(np.isfinite(g)) and np.all(g >= 0)
    mu = max_ulp(g, o)
    assert mu <= ulp, (dist, engine, params, n, mu)
    return mu


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("alpha", [0.1, 0.3, 1.0, 2.5, 30.0])
def test_gamma_parity(engine, alpha):
    ulp = 0 if alpha >= 1 else 2
    for n in SIZES:
        check("gamma", engine, 7, n, (alpha,), ulp)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("ab", [(0.5, 0.5), (2.0, 5.0)])
def test_beta_parity(engine, ab):
    ulp = 0 if min(ab) >= 1 else BOOST_ULP["beta"]
    for n in SIZES:
        check("beta", engine, 7, n, ab, ulp)


def test_gamma_positions_and_continuation():
    for pos, stream in [(1, None), (12345, 3), (2 ** 40 + 7, None)]:
        check("gamma", "xoshiro256pp", 9, 30_000, (2.5,), 0, pos=pos, stream=stream)
    a, p1 = gpu_fill("gamma", "philox4x32_10", 3, None, 0, 5000, (0.3,))
    b, p2 = gpu_fill("gamma", "philox4x32_10", 3, None, p1, 7000, (0.3,))
    c, p3 = gpu_fill("gamma", "philox4x32_10", 3, None, 0, 12000, (0.3,))
    assert p2 == p3 and np.array_equal(np.concatenate([a, b]).view(np.uint64), c.view(np.uint64))


def test_gamma_full_size_sampled():
    """Workload size n = 2^26 (gamma alpha = 2.5 and 0.3, beta (2,5)):
    whole-array compare against the oracle and identical consumed words."""
    for dist, params, ulp in [("gamma", (2.5,), 0), ("gamma", (0.3,), 2), ("beta", (2.0, 5.0), 0)]:
        check(dist, "xoshiro256pp", 7, 1 << 26, params, ulp)
