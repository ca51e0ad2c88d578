"""The library's correctly rounded log (fast table path with Ziv's rounding
test, double-double fallback) against the oracle's correctly rounded log on
the arguments the samplers give it: 53-bit uniforms U, 1 - U, their
extremes, values just below 1 and the table boundaries.  Likewise its
correctly rounded exp on the wedge tests' arguments."""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_05099_gb300 as rp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _args():
    rng = np.random.default_rng(17)
    k = rng.integers(1, 2**53, 200000, dtype=np.uint64)
    u = k.astype(np.float64) * 2.0**-53                 # exact: k < 2^53
    near1 = 1.0 - rng.integers(1, 2**20, 20000).astype(np.float64) * 2.0**-53
    small = np.ldexp(1.0, -rng.integers(1, 54, 2000).astype(np.int64)) * (1 + rng.random(2000))
    bounds = []
    for j in range(1024):   # table boundaries of the top 10 mantissa bits, at several exponents
        for e in (-1, -2, -7, -30):
            m = 1.0 + j / 1024.0
            bounds += [np.ldexp(m, e), np.ldexp(np.nextafter(m, 2.0), e), np.ldexp(np.nextafter(m, 0.0), e)]
    x = np.concatenate([u, 1.0 - u, near1, small, np.array(bounds), [2.0**-53, 1.0 - 2.0**-53, 0.5, 0.25]])
    return x[(x > 0) & (x < 1)]


def test_log_cr_matches_oracle():
    x = _args()
    y = rp.rp_log_cr(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = np.array([oracle.cr_log(float(v)) for v in x])
    bad = np.nonzero(y.view(np.int64) != ref.view(np.int64))[0]
    assert len(bad) == 0, (len(bad), x[bad[:5]], y[bad[:5]], ref[bad[:5]])


def test_log_cr_special_values():
    x = torch.tensor([1.0, 0.5, 2.0**-53], dtype=torch.float64, device="cuda")
    y = rp.rp_log_cr(x).cpu().numpy()
    assert y[0] == 0.0
    assert y[1] == oracle.cr_log(0.5) and y[2] == oracle.cr_log(2.0**-53)


def _exp_args():
    """Arguments of the wedge decisions: t = -x^2/2 for normal x in (0, R]
    and t = -x for exponential x in (0, R_exp], plus tiny |t|, exact
    multiples of ln 2 / 2^k and the ends of both ranges."""
    rng = np.random.default_rng(23)
    rn, re = oracle.zig_table(0)[3], oracle.zig_table(1)[3]
    xn = rng.random(100000) * rn
    xe = rng.random(100000) * re
    tiny = -np.ldexp(1.0, -rng.integers(1, 60, 2000).astype(np.int64)) * (1 + rng.random(2000))
    ln2 = np.log(2.0)
    steps = -np.array([k * ln2 / 2.0 ** j for j in (0, 1, 8) for k in range(1, 20)])
    t = np.concatenate([-0.5 * xn * xn, -xe, tiny, steps, [-0.5 * rn * rn, -re, -0.0, -2.0**-1074]])
    return t[t >= -0.5 * rn * rn - 1.0]


def test_exp_cr_matches_oracle():
    """The library's correctly rounded exp (double-double evaluation) against
    the oracle's, bit for bit, on the wedge tests' arguments."""
    t = _exp_args()
    y = rp.rp_exp_cr(torch.tensor(t, device="cuda")).cpu().numpy()
    ref = np.array([oracle.cr_exp(float(v)) for v in t])
    bad = np.nonzero(y.view(np.int64) != ref.view(np.int64))[0]
    assert len(bad) == 0, (len(bad), t[bad[:5]], y[bad[:5]], ref[bad[:5]])
