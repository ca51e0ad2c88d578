"""Host model of the Philox one-word kernel's index arithmetic (k_onepw_ctr
in csrc/rp_fill_impl.cuh): thread g of a grid of G threads takes blocks
b_first + g, b_first + g + G, ..., block B holds stream words 2B and 2B + 1
(Philox4x32-10 packs two 64-bit words per 128-bit block), and output i is
stream word w0 + i.  For every parity of w0, every 8-byte offset of the
output and grids smaller and larger than the block count, each output must
be written exactly once, with the word it stands for, by a 16-byte store
only where the address is 16-byte aligned.  A check of the kernel's method
on the host, not of the oracle."""
import itertools

import pytest


def model(w0, n, out_addr, G):
    writes = {}
    wide = 0
    b_first = w0 >> 1
    nb = ((w0 + n - 1) >> 1) - b_first + 1
    pairs = (((out_addr >> 3) + w0) & 1) == 0
    for g in range(G):
        j = g
        while j < nb:
            B = b_first + j
            p0 = 2 * B - w0
            words = (2 * B, 2 * B + 1)
            if pairs and p0 >= 0 and p0 + 1 < n:
                assert (out_addr + 8 * p0) % 16 == 0
                wide += 1
                for h in range(2):
                    writes.setdefault(p0 + h, []).append(words[h])
            else:
                for h in range(2):
                    p = p0 + h
                    if 0 <= p < n:
                        writes.setdefault(p, []).append(words[h])
            j += G
    return writes, wide


@pytest.mark.parametrize("w0,n,addr,G", list(itertools.product(
    [0, 1, 2, 7, 12345, 2 ** 40 + 1], [1, 2, 3, 64, 1023], [0, 8, 16, 24], [1, 5, 128, 4096])))
def test_every_output_once_with_its_word(w0, n, addr, G):
    writes, wide = model(w0, n, addr, G)
    assert sorted(writes) == list(range(n))
    for i, ws in writes.items():
        assert ws == [w0 + i]
    if n >= 4:
        # the aligned case stores pairs for all but at most the two ends
        aligned = (((addr >> 3) + w0) & 1) == 0
        assert (wide >= (n - 2) // 2) if aligned else wide == 0
