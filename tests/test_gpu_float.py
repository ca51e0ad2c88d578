"""GPU parity of the float variants (Table "continuous", suffix f; the stream
read as 32-bit words, low half first) against the oracle's float samplers,
through the C ABI: every output bit for bit and the same consumed words, on
all engines, over sizes that span many tiles with ragged ends, from odd and
even start words; fills split over several launches (which then resume in
the middle of a word); asynchronous positions; and the argument checks."""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_05099_gb300 as rp

pytestmark = pytest.mark.gpu

ENGINES = ["xoshiro256pp", "pcg64dxsm", "philox4x32_10", "philox4x64_10", "xoshiro256ss"]
FILL = {"uniformf": rp.rp_fill_uniformf, "normalf": rp.rp_fill_normalf, "expf": rp.rp_fill_expf}


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rp.rp_debug_faults("clear")
    yield
    rp.rp_debug_faults("clear")


def _gpu(dist, engine, seed, pos, n, stream=rp.NO_STREAM):
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    p = FILL[dist](engine, seed, stream, pos, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), p


def _check(dist, engine, seed, pos, n, stream=None):
    got, gpos = _gpu(dist, engine, seed, pos, n, rp.NO_STREAM if stream is None else stream)
    g = oracle.gen(engine, seed, stream, pos=pos)
    ref = oracle.fill(g, dist, n)
    assert gpos == int(g.pos), (dist, engine, n, gpos, int(g.pos))
    bad = np.nonzero(got.view(np.uint32) != ref.view(np.uint32))[0]
    assert len(bad) == 0, (dist, engine, n, bad[:5], got[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("dist", list(FILL))
def test_float_parity(engine, dist):
    for n, pos in ((1, 0), (2, 7), (3, 1), (1023, 12345), (100_003, 2 ** 40 + 1), (1 << 20, 3)):
        _check(dist, engine, 2024, pos, n)


@pytest.mark.parametrize("dist", ["normalf", "expf"])
def test_float_full_size(dist):
    """2^26 outputs from one stream (many tiles, thousands of tails)."""
    _check(dist, "xoshiro256pp", 7, 0, 1 << 26)


@pytest.mark.parametrize("dist", ["normalf", "expf"])
def test_float_fill_split_over_launches(dist):
    """Launches of two tiles each: every continuation starts where the chain
    stopped, in the middle of a word when it stopped on a low half."""
    rp.rp_debug_faults("tile_cap", 2)
    for n, pos in ((300_001, 5), (123_457, 0)):
        _check(dist, "philox4x32_10", 31, pos, n)
        _check(dist, "xoshiro256pp", 32, pos, n)


@pytest.mark.parametrize("dist", list(FILL))
def test_float_async_position(dist):
    n = 200_001
    ref, pos = _gpu(dist, "pcg64dxsm", 5, 17, n)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    pp = torch.empty(1, dtype=torch.int64).pin_memory()
    pp[0] = 17
    FILL[dist]("pcg64dxsm", 5, rp.NO_STREAM, pp, out)
    torch.cuda.synchronize()
    rp.rp_async_status()
    assert int(pp[0]) == pos
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_float_argument_checks():
    buf = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RPError) as ei:
        rp.rp_fill_uniformf("xoshiro256pp", 1, rp.NO_STREAM, 0, buf[1:9])   # 4 mod 8
    assert ei.value.code == -2
    # the samplers accept any 4-byte aligned output and write only their n floats
    buf.fill_(7.0)
    rp.rp_fill_normalf("xoshiro256pp", 1, rp.NO_STREAM, 0, buf[1:6])
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert h[0] == 7.0 and np.all(h[6:] == 7.0)
    ref = oracle.fill(oracle.gen("xoshiro256pp", 1, None), "normalf", 5)
    assert np.array_equal(h[1:6].view(np.uint32), ref.view(np.uint32))
    assert rp.rp_fill_expf("xoshiro256pp", 1, rp.NO_STREAM, 3, buf[:0]) == 3
