"""Pins of the oracle's engines, seeding and jumps against things other than
the oracle itself: NumPy's SeedSequence / PCG64DXSM run as black boxes, jump
identities with two independent jump constructions (Sec. 4.4), and
statistics.  Philox4x32-10 is pinned bit-for-bit against cuRAND in the GPU
suite (tests/test_gpu_fills.py, test_philox_bijection_matches_curand); on
the CPU only its structural properties are checked here.  xoshiro256++'s
transition is pinned by its primitive characteristic polynomial and the
jump identities, but its "++" output function has no external pin: no
published test vectors are on this machine and NumPy has no xoshiro, so
the scrambler's parity is unpinned (its bit balance is checked only)."""
import ctypes
import json
import os

import numpy as np
import pytest
from numpy.random import PCG64DXSM, SeedSequence


def _rng():
    return np.random.default_rng(20240601)


def _gold_engines():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_engines.json")) as f:
        return json.load(f)


def _table_period(engine):
    """Period printed in Table "engines", as an integer."""
    form = _gold_engines()[engine]["period_log2_form"]
    base, _, rest = form.partition("^")
    exp, _, minus = rest.partition("-")
    return int(base) ** int(exp) - (int(minus) if minus else 0)


# ------------------------------------------------------------------ seeding
def test_seedseq_matches_numpy(orc):
    """Sec. 2.3: seed + spawn key -> 128-bit pool -> state words; reading =
    NumPy SeedSequence semantics.  10^4 random (seed, key) pairs plus edges."""
    rng = _rng()
    seeds = [0, 1, 2 ** 32 - 1, 2 ** 32, 2 ** 64 - 1] + [int(x) for x in rng.integers(0, 2 ** 63, 10_000)]
    keys = [None, 0, 1, 2 ** 32, 2 ** 64 - 1] + [int(x) for x in rng.integers(0, 2 ** 40, 10_000)]
    for i, seed in enumerate(seeds):
        key = keys[i % len(keys)]
        ss = SeedSequence(seed) if key is None else SeedSequence(seed, spawn_key=(key,))
        ref = ss.generate_state(12, np.uint32)
        got = orc.seedseq_generate(orc.seedseq_entropy(seed, key), 12)
        assert np.array_equal(ref, got), (seed, key)


def test_xoshiro_seed_is_seedseq_words(orc):
    for seed, key in [(12345, None), (2024, None), (7, 1), (99, None)]:
        g = orc.gen("xoshiro256pp", seed, key)
        ss = SeedSequence(seed) if key is None else SeedSequence(seed, spawn_key=(key,))
        assert orc.state_words(g) == [int(x) for x in ss.generate_state(4, np.uint64)]


# ------------------------------------------------------------------ PCG64
@pytest.mark.parametrize("seed,key", [(0, None), (2024, None), (12345, 3), (2 ** 63 + 11, None)])
def test_pcg64dxsm_matches_numpy(orc, seed, key):
    """Sec. 2.2 / Sec. 5.1: pcg64 is validated against NumPy.  Seeded state,
    increment and the first 10^6 words must be identical."""
    ss = SeedSequence(seed) if key is None else SeedSequence(seed, spawn_key=(key,))
    bg = PCG64DXSM(ss)
    g = orc.gen("pcg64dxsm", seed, key)
    s = orc.state_words(g)
    st = bg.state["state"]
    assert st["state"] == (s[0] << 64 | s[1]) and st["inc"] == (s[2] << 64 | s[3])
    assert np.array_equal(bg.random_raw(1_000_000), orc.next_words(g, 1_000_000))


def test_pcg64dxsm_advance_matches_numpy(orc):
    """Sec. 2.3: PCG64 advance by an arbitrary delta (LCG skip-ahead)."""
    rng = _rng()
    for _ in range(50):
        delta = int(rng.integers(0, 2 ** 62)) << 66 | int(rng.integers(0, 2 ** 62))
        bg = PCG64DXSM(SeedSequence(5))
        g = orc.gen("pcg64dxsm", 5)
        bg.advance(delta)
        orc.lib().or_jump(ctypes.byref(g), (delta >> 64) & (2 ** 64 - 1), delta & (2 ** 64 - 1))
        assert np.array_equal(bg.random_raw(8), orc.next_words(g, 8))


# ------------------------------------------------------------------ xoshiro
def test_xoshiro_charpoly_primitive_shape(orc):
    """T^N = p_N(T) needs the degree-256 characteristic polynomial
    (Cayley-Hamilton, Sec. 4.4).  Pins: degree 256, constant term 1, and
    x^(2^256 - 1) = 1 mod p (period 2^256 - 1, Table "engines")."""
    p = orc.xoshiro_charpoly()
    assert p.bit_length() - 1 == 256 and (p & 1) == 1

    def mulmod(a, b):
        r = 0
        while b:
            if b & 1:
                r ^= a
            b >>= 1
            a <<= 1
            if (a >> 256) & 1:
                a ^= p
        return r

    def powmod(e):
        r, base = 1, 2
        while e:
            if e & 1:
                r = mulmod(r, base)
            base = mulmod(base, base)
            e >>= 1
        return r

    period = _table_period("xoshiro256pp")
    assert period == 2 ** 256 - 1 and _table_period("xoshiro256ss") == period
    assert powmod(period) == 1
    # x has order exactly 2^256 - 1 (p is primitive): x^(P/q) != 1 for every
    # prime q of P = 2^256 - 1 = F0 F1 ... F7 (Fermat numbers); the list is
    # checked to be the complete factorisation into primes
    primes = (3, 5, 17, 257, 65537, 641, 6700417, 274177, 67280421310721,
              59649589127497217, 5704689200685129054721)
    sympy = pytest.importorskip("sympy")
    prod = 1
    for q in primes:
        assert sympy.isprime(q)
        prod *= q
    assert prod == period
    for q in primes:
        assert powmod(period // q) != 1


def test_xoshiro_jump_equals_steps(orc):
    """jump(N) == N single steps, N <= 4096 plus random N, for both jump
    constructions (polynomial and matrix)."""
    g = orc.gen("xoshiro256pp", 12345)
    s0 = orc.state_words(g)
    words = orc.next_words(g, 4100)
    rng = _rng()
    Ns = [0, 1, 2, 3, 63, 64, 255, 256, 257, 1000, 4095] + [int(x) for x in rng.integers(0, 4096, 6)]
    for N in Ns:
        for method in ("poly", "matrix"):
            s = orc.xoshiro_jump(s0, N, method)
            h = orc.Gen()
            orc.lib().or_gen_set(ctypes.byref(h), 1, np.array(s, np.uint64).ctypes.data_as(ctypes.c_void_p))
            assert int(orc.next_words(h, 1)[0]) == int(words[N]), (N, method)


def test_xoshiro_jump_composition_and_methods_agree(orc):
    """jump(a) o jump(b) == jump(a+b); T^(2^k) by matrix squaring == by the
    jump polynomial for k in {32, 64, 96, 128, 192} (Sec. 2.3)."""
    s0 = orc.state_words(orc.gen("xoshiro256pp", 99))
    rng = _rng()
    for _ in range(4):
        a = int(rng.integers(0, 2 ** 63)) * 3 + 1
        b = int(rng.integers(0, 2 ** 63)) << 40
        assert orc.xoshiro_jump(orc.xoshiro_jump(s0, a), b) == orc.xoshiro_jump(s0, a + b)
    for k in (32, 64, 96, 128, 192):
        assert orc.xoshiro_jump(s0, 2 ** k, "poly") == orc.xoshiro_jump(s0, 2 ** k, "matrix")


def test_xoshiro_bit_balance(orc):
    """Statistics: each of the 64 bit positions is 1 with probability 1/2."""
    g = orc.gen("xoshiro256pp", 2024)
    w = orc.next_words(g, 1 << 18)
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 64).mean(axis=0)
    sigma = 0.5 / np.sqrt(len(w))
    assert np.all(np.abs(bits - 0.5) < 6 * sigma)


def test_seek_matches_sequential(orc):
    for eng in ("xoshiro256pp", "pcg64dxsm", "philox4x32_10"):
        g = orc.gen(eng, 31337)
        w = orc.next_words(g, 3000)
        for p in (0, 1, 2, 777, 2999):
            h = orc.gen(eng, 31337, pos=p)
            assert int(orc.next_words(h, 1)[0]) == int(w[p]), (eng, p)


# ------------------------------------------------------------------ Philox
def test_philox_structure(orc):
    """Counter-based: word p is half (p mod 2) of block counter + p/2; the
    counter is a 128-bit integer (carry across the 32-bit lanes); different
    keys give unrelated blocks; output bits are balanced."""
    g = orc.gen("philox4x32_10", 2024)
    ctr = g.s[0] | (g.s[1] << 64)
    key = g.s[2]
    w = orc.next_words(g, 64)
    for b in range(32):
        c = ctr + b
        o = orc.philox([(c >> (32 * i)) & 0xFFFFFFFF for i in range(4)], [key & 0xFFFFFFFF, key >> 32])
        assert int(w[2 * b]) == o[0] | (o[1] << 32) and int(w[2 * b + 1]) == o[2] | (o[3] << 32)
    # carry propagation across 32-bit lanes
    a = orc.philox([0xFFFFFFFF, 0, 0, 0], [1, 2])
    b = orc.philox([0, 1, 0, 0], [1, 2])
    assert a != b
    outs = np.array([orc.philox([i, 0, 0, 0], [5, 6]) for i in range(4096)], np.uint32)
    bits = np.unpackbits(outs.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 6 * 0.5 / np.sqrt(outs.size * 32)


# ------------------------------------------------------------------ Philox4x64-10
def test_philox4x64_matches_numpy(orc):
    """The paper's Philox (4x64-10) with NumPy's Philox seeding and counter
    convention: key = two SeedSequence words, counter 0, incremented before
    each block; every word equals numpy.random.Philox's random_raw."""
    for seed, key in ((2024, None), (7, 0), (99, 5), (2 ** 63 + 11, 123456789)):
        g = orc.gen("philox4x64_10", seed, key)
        ss = np.random.SeedSequence(seed) if key is None else np.random.SeedSequence(seed, spawn_key=(key,))
        ref = np.random.Philox(ss).random_raw(40_001)
        assert np.array_equal(orc.next_words(g, 40_001), ref), (seed, key)


def test_philox4x64_block_function(orc):
    """Word p is word p mod 4 of the block at counter + 1 + p/4 (a 128-bit
    counter, carry into the second word), through the bijection itself."""
    g = orc.gen("philox4x64_10", 31)
    key = [int(g.s[2]), int(g.s[3])]
    w = orc.next_words(g, 4 * 20)
    for b in range(20):
        assert [int(x) for x in w[4 * b:4 * b + 4]] == orc.philox4x64([b + 1, 0, 0, 0], key)
    assert orc.philox4x64([2 ** 64 - 1, 0, 0, 0], [1, 2]) != orc.philox4x64([0, 1, 0, 0], [1, 2])


def test_philox4x64_seek_and_substreams(orc):
    g = orc.gen("philox4x64_10", 31337)
    w = orc.next_words(g, 3000)
    for p in (0, 1, 3, 4, 5, 777, 2999):
        h = orc.gen("philox4x64_10", 31337, pos=p)
        assert int(orc.next_words(h, 1)[0]) == int(w[p]), p
    base = orc.state_words(orc.gen("philox4x64_10", 99))
    for s in (0, 1, 4095):
        st = orc.state_words(orc.substream("philox4x64_10", 99, s))
        assert st == [0, 0, s, base[3]], s


def test_uniform52_closed_form(orc):
    """Sec. 3.1 method 2 (the paper's default): the word's top 52 bits in the
    fraction of a double in [1, 2), minus 1, is exactly floor(u/2^12) 2^-52."""
    w = orc.next_words(orc.gen("philox4x64_10", 5), 1 << 16)
    u = orc.fill(orc.gen("philox4x64_10", 5), "uniform52", 1 << 16)
    assert np.array_equal((u * 2.0 ** 52).astype(np.uint64), w >> np.uint64(12))
    assert u.min() >= 0.0 and u.max() < 1.0


# ------------------------------------------------------------------ xoshiro256**
def _unscramble_ss(w):
    """Inverse of the xoshiro256** scrambler x -> rotl(5 x, 7) 9 (mod 2^64):
    multiply by the inverse of 9, rotate right by 7, multiply by the inverse
    of 5.  The inverses come from Python's modular arithmetic, so a scrambler
    that read another state word, or applied its steps in another order,
    would not come back to the state."""
    M = 2 ** 64
    y = (int(w) * pow(9, -1, M)) % M
    y = ((y >> 7) | (y << 57)) % M
    return (y * pow(5, -1, M)) % M


def test_xoshiro256ss_outputs_recover_the_shared_state(orc):
    """Table "engines": xoshiro256** and xoshiro256++ share the seeding and
    the linear transition and differ only in the scrambler.  Stepping the
    xoshiro256++ generator (whose transition is pinned by its characteristic
    polynomial and jump identities) gives the state word s1 before each
    step; every xoshiro256** output, unscrambled, must equal it."""
    for seed, key in [(2024, None), (7, 3)]:
        pp = orc.gen("xoshiro256pp", seed, key)
        ss = orc.gen("xoshiro256ss", seed, key)
        assert orc.state_words(pp) == orc.state_words(ss)
        for _ in range(2000):
            s1 = orc.state_words(pp)[1]
            orc.next_words(pp, 1)
            assert _unscramble_ss(orc.next_words(ss, 1)[0]) == s1


def test_xoshiro256ss_jumps_seek_and_substreams(orc):
    """The jump polynomial is the transition's, so it serves both engines:
    seeking equals stepping, and substream s starts from the xoshiro256++
    substream's state."""
    g = orc.gen("xoshiro256ss", 31337)
    w = orc.next_words(g, 3000)
    for p in (0, 1, 2, 777, 2999):
        h = orc.gen("xoshiro256ss", 31337, pos=p)
        assert int(orc.next_words(h, 1)[0]) == int(w[p]), p
    for s in (0, 1, 4095):
        assert orc.state_words(orc.substream("xoshiro256ss", 99, s)) == orc.state_words(orc.substream("xoshiro256pp", 99, s))


def test_xoshiro256ss_bit_balance(orc):
    w = orc.next_words(orc.gen("xoshiro256ss", 2024), 1 << 18)
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 64).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 6 * 0.5 / np.sqrt(len(w)))


def test_engine_table_state_words_and_pcg_period(orc):
    """Table "engines" (golden): xoshiro and PCG64-DXSM keep 4 state words
    (the oracle's and the library's layout); PCG64-DXSM has period 2^128 (a
    jump by half the period moves the state, two of them bring it back).
    Philox-4x64 is printed with 6 words (a 256-bit counter and a 128-bit
    key); this library keeps the counter's upper 128 bits at zero, so its
    state is 4 words and a stream has 2^130 words."""
    gold = _gold_engines()
    for eng in ("xoshiro256pp", "xoshiro256ss", "pcg64dxsm"):
        assert gold[eng]["state_words"] == len(orc.state_words(orc.gen(eng, 1)))
    assert gold["philox4x64_10"]["state_words"] == 6
    period = _table_period("pcg64dxsm")
    s0 = orc.state_words(orc.gen("pcg64dxsm", 99))
    half = orc.pcg_advance(s0, period // 2)
    assert half[:2] != s0[:2] and half[2:] == s0[2:]
    assert orc.pcg_advance(half, period // 2) == s0
