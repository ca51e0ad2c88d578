"""Host check of the bit-parallel candidate chain of the ziggurat kernel's
first pass (Sec. 3.1: a candidate is one word when its fast test passes,
else two for a wedge; ties of the top bits count as not fast and tails are
walked separately).  The kernel finds the candidate starts of a 16-word
half-block from the non-fast mask with a few word operations instead of 16
dependent steps; here that mask arithmetic, restated, is compared with the
sequential recurrence on every 16-bit fast mask, every starting position and
both carry-in states, including the carry out of the half-block."""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def _masks(F, frm, ein):
    """The kernel's mask arithmetic (32-bit words; positions 0..15)."""
    rng = np.uint64((0xFFFF << frm) & 0xFFFF)
    e = np.uint64(ein << frm)
    N = ~F & rng
    R = N & ~e
    RS = R & ~((R << np.uint64(1)) & M32)
    Er = R & ~((R + (RS & np.uint64(0x55555555))) & M32)
    Or = R & ~((R + (RS & np.uint64(0xAAAAAAAA))) & M32)
    K = (((Er << np.uint64(1)) & np.uint64(0xAAAAAAAA)) | ((Or << np.uint64(1)) & np.uint64(0x55555555)) | e) & M32
    Sc = ~K & rng
    return Sc, (K >> np.uint64(16)) & np.uint64(1)


def _sequential(F, frm, ein):
    """Walk the words in order: a start that fails the fast test consumes the
    next word as its second word."""
    second = np.full(F.shape, bool(ein))
    Sc = np.zeros(F.shape, np.uint64)
    for q in range(frm, 16):
        fast = ((F >> np.uint64(q)) & np.uint64(1)).astype(bool)
        start = ~second
        Sc |= start.astype(np.uint64) << np.uint64(q)
        second = start & ~fast
    return Sc, second.astype(np.uint64)


def test_chain_masks_equal_the_sequential_walk():
    F = np.arange(1 << 16, dtype=np.uint64)
    for frm in range(16):
        for ein in (0, 1):
            sc, carry = _masks(F, frm, ein)
            sc_ref, carry_ref = _sequential(F, frm, ein)
            assert np.array_equal(sc, sc_ref), (frm, ein)
            assert np.array_equal(carry, carry_ref), (frm, ein)
