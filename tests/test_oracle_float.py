"""Pins of the oracle's float variants (Table "continuous", suffix f;
Sec. 3.1: the stream read as 32-bit words, low half of each 64-bit word
first; Sec. 4.4): the float ziggurat tables against the exact strip
geometry rounded once to float, the uniform's closed form and word order,
and the laws of the float normal and exponential (SciPy CDFs, moments, the
fast-accept fraction the tables imply, the tail mass beyond R)."""
import math
import os
import sys

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", "oracle"))
import gen_ziggurat as gz  # noqa: E402

N = 1 << 20
P_MIN = 1e-4


def _rn_float(x):
    """x rounded once to binary32 (24-bit significand, nearest-even)."""
    with mp.workprec(24):
        return np.float32(float(mp.mpf(x)))


@pytest.mark.parametrize("which,kind,scale", [(0, "normal", 2 ** 23), (1, "exp", 2 ** 24)])
def test_float_tables_are_the_exact_geometry_rounded_once(orc, which, kind, scale):
    """k_i = floor(M x_{i-1} / x_i), w_i = RN_f(x_i / M), f_i = RN_f(f(x_i))
    with M = 2^23 (normal, 23-bit magnitude) or 2^24 (exponential), from the
    60-digit strip construction; the base strip uses q = v / f(R)."""
    t = gz.tables(kind)
    xs, f = t["x"], (gz._normal_f if which == 0 else gz._exp_f)
    k, w, fv = orc.zig_table_f(which)
    assert int(k[0]) == int(mp.floor(scale * t["r"] / t["q"])) and w[0] == _rn_float(t["q"] / scale) and fv[0] == 1.0
    assert int(k[1]) == 0
    for i in range(1, 256):
        if i > 1:
            assert int(k[i]) == int(mp.floor(scale * xs[i - 1] / xs[i])), i
        assert w[i] == _rn_float(xs[i] / scale), i
        assert fv[i] == _rn_float(f(xs[i])), i


def _halves(words):
    h = np.empty(2 * len(words), np.uint64)
    h[0::2] = words & np.uint64(0xFFFFFFFF)
    h[1::2] = words >> np.uint64(32)
    return h


@pytest.mark.parametrize("engine", ["xoshiro256pp", "philox4x32_10", "pcg64dxsm"])
def test_uniformf_closed_form_and_word_order(orc, engine):
    """uniformf of 32-bit word h is floor(h / 2^9) 2^-23 exactly; words are
    the low half of each stream word, then its high half; an odd count
    leaves the last high half unused (the position is the next word)."""
    n = 10_001
    w = orc.next_words(orc.gen(engine, 5, pos=3), (n + 1) // 2)
    g = orc.gen(engine, 5, pos=3)
    u = orc.fill(g, "uniformf", n)
    assert u.dtype == np.float32 and int(g.pos) == 3 + (n + 1) // 2
    h = _halves(w)[:n]
    assert np.array_equal((u.astype(np.float64) * 2.0 ** 23).astype(np.uint64), h >> np.uint64(9))
    assert u.min() >= 0.0 and u.max() < 1.0


@pytest.mark.parametrize("engine", ["xoshiro256pp", "philox4x64_10"])
def test_normalf_and_expf_laws(orc, engine):
    x = orc.fill(orc.gen(engine, 2024), "normalf", N).astype(np.float64)
    assert stats.kstest(x, "norm").pvalue > P_MIN
    assert abs(x.mean()) < 6 / math.sqrt(N) and abs(x.var() - 1.0) < 6 * math.sqrt(2.0 / N)
    e = orc.fill(orc.gen(engine, 2024), "expf", N).astype(np.float64)
    assert stats.kstest(e, "expon").pvalue > P_MIN
    assert abs(e.mean() - 1.0) < 6 / math.sqrt(N) and e.min() >= 0.0


def test_normalf_fast_fraction_and_tail_mass(orc):
    """Each candidate is fast-accepted with probability (1/256) sum_i k_i/2^23
    (r is uniform on 23 bits); outputs beyond R carry the tail mass
    2 (1 - Phi(R)).  Both within 5 binomial sigma."""
    g = orc.gen("xoshiro256pp", 99)
    x = orc.fill(g, "normalf", N)
    c = orc.zig_counts()
    k, _, _ = orc.zig_table_f(0)
    p_fast = float(k.astype(np.float64).sum()) / 256.0 / 2 ** 23
    cand = c["fast"] + c["wedge"] + c["tail"]   # every candidate is fast, a wedge test or a tail
    assert abs(c["fast"] / cand - p_fast) < 5 * math.sqrt(p_fast * (1 - p_fast) / cand)
    R = orc.zig_table(0)[3]
    p_tail = 2 * stats.norm.sf(R)
    frac = np.mean(np.abs(x.astype(np.float64)) > R)
    assert abs(frac - p_tail) < 5 * math.sqrt(p_tail / N) + 1e-7


def test_float_fills_start_on_word_boundaries(orc):
    """A float fill starts at the low half of word pos (accepted candidates
    begin at 32-bit word 2 pos or later, in increasing order), and the next
    fill starts at the low half of the word after the last one read."""
    g = orc.gen("xoshiro256pp", 31, pos=7)
    a, start = orc.fill(g, "normalf", 1001, with_start=True)
    assert int(start[0]) >= 14 and np.all(np.diff(start.astype(np.int64)) > 0)
    p = int(g.pos)
    assert 2 * p >= int(start[-1]) + 1
    b, s2 = orc.fill(g, "normalf", 5, with_start=True)
    assert int(s2[0]) >= 2 * p
    # the same values as a fresh generator started at word p
    c = orc.fill(orc.gen("xoshiro256pp", 31, pos=p), "normalf", 5)
    assert np.array_equal(b.view(np.uint32), c.view(np.uint32))
