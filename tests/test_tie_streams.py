"""Host checks of the near-tie stream construction (tests/tie_streams.py),
against the oracle alone: the Philox4x32-10 inverse undoes the oracle's
block function, the chosen words appear at the chosen positions, and each
constructed decision lands at its tie in both outcomes (Sec. 3.1 samplers,
decided with the oracle's correctly rounded exp and log)."""
import numpy as np

import oracle
from tie_streams import (M32, block, mt_ties, oracle_gen, philox_inverse, state_with_block, tail_pair_ties,
                         wedge_ties)


def test_philox_inverse_undoes_the_block_function():
    rng = np.random.default_rng(9)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 1 << 32, 4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 1 << 32, 2, dtype=np.uint64)]
        assert philox_inverse(oracle.philox(ctr, key), key) == ctr


def test_chosen_words_lead_the_stream():
    rng = np.random.default_rng(10)
    for _ in range(20):
        w0, w1, key = (int(x) for x in rng.integers(0, 1 << 63, 3, dtype=np.uint64))
        words = state_with_block(w0, w1, key)
        assert [int(x) for x in oracle.next_words(oracle_gen(words), 2)] == [w0, w1]
        c = words[0] | (words[1] << 64)
        assert block(c, key) == (w0, w1) and block(c + 1, key)[0] & M32 == int(oracle.next_words(oracle_gen(words), 3)[2]) & M32


def _first(dist, words, pos, n, *p):
    g = oracle_gen(words)
    if pos:
        oracle.next_words(g, pos)
    return oracle.fill(g, dist, n, *p, with_start=True)[1]


def test_wedge_ties_reach_both_outcomes():
    for expo in (False, True):
        cases = wedge_ties(expo, np.random.default_rng(5), (1, 128))
        firsts = [int(_first("exp" if expo else "normal", w, p, 4)[0]) == 0 for w, p in cases]
        assert set(firsts) == {True, False}


def test_tail_pair_ties_reach_both_outcomes():
    cases = tail_pair_ties(np.random.default_rng(6), 2)
    lens = [int(_first("normal", w, p, 2)[1]) - 1 for w, p in cases]
    assert 3 in lens and any(x > 3 for x in lens), lens


def test_mt_ties_reach_both_outcomes():
    for alpha in (2.5, 0.3):
        cases = mt_ties(alpha, np.random.default_rng(7), 2)
        firsts = [int(_first("gamma", w, p, 2, alpha)[0]) == 0 for w, p in cases]
        assert set(firsts) == {True, False}, (alpha, firsts)
