"""GPU parity at chunk seams, where a candidate or a variate that started in
one thread's chunk reaches into the next (Sec. 3.1 samplers; the seams are
this library's).  The streams come from host models of the seam rules
(tests/test_merge_points.py): an 11-word normal tail across a seam of the
ziggurat kernel, and beta shapes whose gamma draws leave runs of chunks
without a merge point."""
import pytest
import torch

from gpu_util import assert_parity
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
    """Shapes whose gamma draws mostly consume the same word counts leave
    runs of chunks without a merge point: on this stream the longest runs
    are 14 chunks (2, 2.01) and 8 chunks (10, 11), per the host model of the
    merge rule.  A walk crosses them (up to 64), and the fill stays
    bit-exact."""
    check("beta", "philox4x32_10", 7, 1 << 18, ab, 0)
