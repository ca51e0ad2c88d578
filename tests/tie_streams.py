"""Streams built around near-ties of the exact accept decisions (Sec. 3.1
samplers; Sec. 4.2 exactness), for GPU parity tests.

The decisions are first taken in FP32 with a proven margin, then in FP64
with libm and a margin of its error, and only then with correctly rounded
exp/log.  Random words reach the last stage almost never, so the streams
here place chosen words at a decision: Philox4x32-10's block function is a
bijection of the 128-bit counter for a fixed key (each round's products by
odd constants are invertible mod 2^32), so any two chosen words are block 0
of the stream whose state (counter, key) is the inverse image.  A fill from
those state words (rp_fill_state, and the oracle's generator set to the same
words) then meets the chosen candidate first.  The tie values come from the
oracle's correctly rounded exp and log, in the sampler's own evaluation
order.  Nothing here comes from the CUDA path."""
import math

import numpy as np

import oracle

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
M52 = (1 << 52) - 1
PH_M0, PH_M1 = 0xD2511F53, 0xCD9E8D57      # Philox4x32 multipliers
PH_W0, PH_W1 = 0x9E3779B9, 0xBB67AE85      # key increments per round
PH_M0_INV, PH_M1_INV = pow(PH_M0, -1, 1 << 32), pow(PH_M1, -1, 1 << 32)


def philox_inverse(out4, key2):
    """Counter (four 32-bit lanes) whose Philox4x32-10 block under key2 is
    out4: the ten rounds undone from the last."""
    x0, x1, x2, x3 = out4
    k0, k1 = key2
    for r in reversed(range(10)):
        ka, kb = (k0 + r * PH_W0) & M32, (k1 + r * PH_W1) & M32
        y0, y1, y2, y3 = x0, x1, x2, x3
        x2 = (y1 * PH_M1_INV) & M32
        x1 = y0 ^ ((PH_M1 * x2) >> 32) ^ ka
        x0 = (y3 * PH_M0_INV) & M32
        x3 = y2 ^ ((PH_M0 * x0) >> 32) ^ kb
    return [x0, x1, x2, x3]


def words_to_lanes(w0, w1):
    """Block lanes of two stream words (word = x0 | x1 << 32, x2 | x3 << 32)."""
    return [w0 & M32, w0 >> 32, w1 & M32, w1 >> 32]


def lanes_to_words(x):
    return x[0] | (x[1] << 32), x[2] | (x[3] << 32)


def state_with_block(w0, w1, key):
    """Philox4x32-10 state words (counter lo, counter hi, key) of a stream
    whose block 0 (words 0 and 1) is (w0, w1)."""
    c = philox_inverse(words_to_lanes(w0, w1), [key & M32, key >> 32])
    c_lo, c_hi = lanes_to_words(c)
    return [c_lo, c_hi, key, 0]


def block(counter128, key):
    """The two stream words of the block at a 128-bit counter value."""
    lanes = [(counter128 >> (32 * j)) & M32 for j in range(4)]
    return lanes_to_words(oracle.philox(lanes, [key & M32, key >> 32]))


def oracle_gen(words):
    g = oracle.Gen()
    g.engine = oracle.ENGINES["philox4x32_10"]
    for i, w in enumerate(words):
        g.s[i] = w
    return g


def u53(k):
    return k * 2.0 ** -53


def zig_word(i, r, sign, top, exponential):
    """Ziggurat candidate word: strip i in bits 0-7, then the sign bit (normal)
    and r (52 bits), or r (53 bits) for the exponential; `top` fills the
    unused high bits."""
    if exponential:
        return (top << 61) | (r << 8) | i
    return (top << 61) | (r << 9) | (sign << 8) | i


def flip(k_lo, k_hi, pred):
    """Adjacent (k_false, k_true) in [k_lo, k_hi] where the monotone predicate
    pred changes value (bisection), or None if it does not change there."""
    a, b = pred(k_lo), pred(k_hi)
    if a == b:
        return None
    lo, hi = k_lo, k_hi          # pred(lo) == a, pred(hi) == b
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if pred(mid) == a:
            lo = mid
        else:
            hi = mid
    return (hi, lo) if a else (lo, hi)


def wedge_ties(exponential, rng, strips):
    """(state words, pos) of streams whose first candidate is a wedge test
    of strip i decided within one ulp of exp(t): for each strip, the U that
    gives y just below exp(t) (accepted) and at or just above it (rejected)."""
    k, w, f, _ = oracle.zig_table(1 if exponential else 0)
    cases = []
    for i in strips:
        ki = int(k[i])
        rmax = (1 << 53) if exponential else (1 << 52)
        for _ in range(50):
            r = ki + int(rng.integers(0, rmax - ki))
            x = float(r) * float(w[i])
            t = -x if exponential else -0.5 * (x * x)
            E = oracle.cr_exp(t)
            d = float(f[i - 1]) - float(f[i])
            res = flip(0, (1 << 53) - 1, lambda kk: d * u53(kk) + float(f[i]) < E)
            if res:
                break
        assert res, ("no tie found", i)
        for kk in res:
            u0 = zig_word(i, r, int(rng.integers(0, 2)), int(rng.integers(0, 8)), exponential)
            u1 = (kk << 11) | int(rng.integers(0, 1 << 11))
            cases.append((state_with_block(u0, u1, int(rng.integers(0, 1 << 63))), 0))
    return cases


def tail_pair_ties(rng, count):
    """(state words, pos) of normal streams whose first candidate (word 1) is
    a tail whose first pair (block 1: words 2 and 3) is decided within one
    ulp of 2b = a^2, a = -log(1 - U1)/R, b = -log(1 - U2), both outcomes.
    The pair's block is chosen; keys are drawn until the word before it is a
    tail candidate (strip 0, not a fast accept: about one key in 4000)."""
    k, _, _, R = oracle.zig_table(0)
    k0 = int(k[0])
    cases = []
    while len(cases) < count:
        # U1 in [0.85, 0.999): a^2 >= 0.27, so that one step of U2 moves 2b by
        # less than 2^-48 of the sides and the tie reaches the correctly
        # rounded stage as well as the libm one
        k1 = int(rng.integers(int(0.85 * 2.0 ** 53), int(0.999 * 2.0 ** 53)))
        a = -oracle.cr_log(1.0 - u53(k1)) / R
        A2 = a * a
        res = flip(0, (1 << 53) - 1, lambda kk: (-oracle.cr_log(1.0 - u53(kk))) * 2.0 > A2)
        if not res:
            continue
        for kk in res:
            w1 = (k1 << 11) | int(rng.integers(0, 1 << 11))
            w2 = (kk << 11) | int(rng.integers(0, 1 << 11))
            for _ in range(200000):
                key = int(rng.integers(0, 1 << 63)) | (int(rng.integers(0, 2)) << 63)
                c1 = philox_inverse(words_to_lanes(w1, w2), [key & M32, key >> 32])
                c1 = c1[0] | (c1[1] << 32) | (c1[2] << 64) | (c1[3] << 96)
                c0 = (c1 - 1) % (1 << 128)
                _, u0 = block(c0, key)
                if (u0 & 0xFF) == 0 and ((u0 >> 9) & M52) >= k0:
                    cases.append(([c0 & M64, c0 >> 64, key, 0], 1))
                    break
    return cases


def mt_params(alpha):
    s = alpha if alpha >= 1.0 else alpha + 1.0
    d = s - 1.0 / 3.0
    return d, 1.0 / math.sqrt(9.0 * d)


def mt_ties(alpha, rng, count):
    """(state words, pos) of gamma streams whose first attempt (a fast normal
    word x, then the uniform U) fails the squeeze U < 1 - 0.0331 x^4 and is
    decided by log U < x^2/2 + d (1 - v + log v) within one ulp, both
    outcomes (Marsaglia-Tsang, Sec. 3.1)."""
    d, c = mt_params(alpha)
    kt, w, _, _ = oracle.zig_table(0)
    cases = []
    tries = 0
    while len(cases) < count:
        tries += 1
        assert tries < 100000
        i = int(rng.integers(2, 256))               # strip 1 has no fast region
        r = int(rng.integers(0, int(kt[i])))        # fast: a one-word normal
        sign = int(rng.integers(0, 2))
        x = float(r) * float(w[i])
        x = -x if sign else x
        v = 1.0 + c * x
        if v <= 0.0:
            continue
        v = v * v * v
        x2 = x * x
        squeeze = 1.0 - 0.0331 * (x2 * x2)
        rhs = 0.5 * x2 + d * ((1.0 - v) + oracle.cr_log(v))
        U = oracle.cr_exp(rhs)
        if not (squeeze < U < 1.0):
            continue
        res = flip(1, (1 << 53) - 1, lambda kk: oracle.cr_log(u53(kk)) < rhs)
        if not res or min(res) * 2.0 ** -53 <= squeeze:
            continue
        for kk in res:
            u0 = zig_word(i, r, sign, int(rng.integers(0, 8)), False)
            u1 = (kk << 11) | int(rng.integers(0, 1 << 11))
            cases.append((state_with_block(u0, u1, int(rng.integers(0, 1 << 63))), 0))
    return cases
