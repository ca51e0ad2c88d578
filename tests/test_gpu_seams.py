"""GPU parity at chunk seams, where a candidate or a variate that started in
one thread's chunk reaches into the next (Sec. 3.1 samplers; the seams are
this library's).  The streams come from host models of the seam rules
(tests/test_merge_points.py): an 11-word normal tail across a seam of the
ziggurat kernel, and beta shapes whose gamma draws leave runs of chunks
without a merge point.  Beta shapes whose two gamma draws almost never
differ in word count leave only phased merge points (chains one gamma
apart); those fills must be exact too."""
import pytest
import torch

from gpu_util import BOOST_ULP, assert_parity
from test_gpu_gamma import check
from test_merge_points import LONG_TAILS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("w", LONG_TAILS)
def test_normal_tail_across_a_chunk_seam(w):
    """An 11-word normal tail (four rejected pairs) on the last word of a
    384-word chunk overhangs the seam by ten words: the fill from 383 words
    before it (first seam) and from 10 chunks further back (a seam between
    two later threads) must still equal the oracle, with the same consumed
    words."""
    for before in (383, 383 + 10 * 384):
        assert_parity("normal", "xoshiro256pp", 2024, None, w - before, 6000)


@pytest.mark.parametrize("ab", [(2.0, 2.01), (10.0, 11.0)])
def test_beta_with_shapes_that_merge_rarely(ab):
    """Shapes whose gamma draws mostly consume the same word counts (under
    the unphased rule these left runs of up to 14 chunks without a merge
    point on this stream): the fill stays bit-exact."""
    check("beta", "philox4x32_10", 7, 1 << 18, ab, 0)


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10"])
@pytest.mark.parametrize("ab", [(2.0, 2.0000001), (30.0, 31.0), (100.0, 100.5), (0.5, 0.5000001), (5.0, 5.0 + 2 ** -40)])
def test_beta_with_shapes_that_consume_alike(engine, ab):
    """Shapes whose gamma draws almost never differ in word count: a chain
    that enters a chunk one gamma later than another stays one gamma apart,
    so the seams are phased merge points (either phase may enter) and the
    walks carry a map from entry to exit phase.  Over many tiles, and from a
    position inside the stream, the fill equals the oracle (bit for bit; the
    boost bar below shape 1) with the same consumed words."""
    ulp = 0 if min(ab) >= 1 else BOOST_ULP["beta"]
    check("beta", engine, 7, 1 << 20, ab, ulp)
    check("beta", engine, 11, 100_003, ab, ulp, pos=12345)
