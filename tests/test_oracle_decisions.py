"""Exactness of the oracle's accept decisions (Sec. 4.2: results must not
depend on the platform's libm; the reading is that every accept test is
the exact comparison).  A plain Python walk over the same words, following
the paper's candidate layout (Sec. 3.1: strip byte, sign bit, magnitude;
one word for a fast accept, a second word for a wedge, pairs of uniforms
for the normal tail), decides every wedge and tail with 40-digit mpmath
values instead of the oracle's double-double functions.  The outputs and
the word that began each accepted candidate must agree exactly, for the
double samplers and their float variants."""
import mpmath as mp
import numpy as np
import pytest

N = 20_000


class _Words:
    """Words of a stream from position 0: 64-bit (double samplers) or the
    32-bit halves, low half first (float variants)."""

    def __init__(self, orc, engine, seed, halves):
        w = orc.next_words(orc.gen(engine, seed), 4 * N)
        if halves:
            h = np.empty(2 * len(w), np.uint64)
            h[0::2] = w & np.uint64(0xFFFFFFFF)
            h[1::2] = w >> np.uint64(32)
            w = h
        self.w = [int(x) for x in w]
        self.p = 0

    def next(self):
        self.p += 1
        return self.w[self.p - 1]


def _log(x):
    with mp.workdps(40):
        return float(mp.log(mp.mpf(x)))   # rounded to nearest from 40 digits


def _below_exp(y, t):
    """y < exp(t) for doubles y and t (t exact as given), on 40 digits."""
    with mp.workdps(40):
        return mp.mpf(y) < mp.exp(mp.mpf(t))


def _below_exp_half_square(y, x):
    """y < exp(-x^2 / 2) with x^2 exact, on 40 digits."""
    with mp.workdps(40):
        xm = mp.mpf(float(x))
        return mp.mpf(float(y)) < mp.exp(-xm * xm / 2)


def _walk_double(orc, words, normal):
    k, w, f, R = orc.zig_table(0 if normal else 1)
    k = [int(v) for v in k]
    out, start = [], []
    while len(out) < N:
        p0 = words.p
        u = words.next()
        i = u & 0xFF
        r = (u >> 9) & (2 ** 52 - 1) if normal else (u >> 8) & (2 ** 53 - 1)
        x = float(r) * w[i]
        if normal and (u >> 8) & 1:
            x = -x
        if r < k[i]:
            out.append(x), start.append(p0)
            continue
        if i == 0:
            if normal:
                while True:
                    a = -_log(1.0 - (words.next() >> 11) * 2.0 ** -53) / R
                    b = -_log(1.0 - (words.next() >> 11) * 2.0 ** -53)
                    if b + b > a * a:
                        break
                v = R + a
                out.append(-v if (u >> 8) & 1 else v), start.append(p0)
            else:
                out.append(R - _log(1.0 - (words.next() >> 11) * 2.0 ** -53)), start.append(p0)
            continue
        U = (words.next() >> 11) * 2.0 ** -53
        y = (f[i - 1] - f[i]) * U + f[i]
        t = -0.5 * (x * x) if normal else -x
        if _below_exp(y, t):
            out.append(x), start.append(p0)
    return np.array(out), np.array(start, np.uint64)


def _walk_float(orc, words, normal):
    k, w, f = orc.zig_table_f(0 if normal else 1)
    R = orc.zig_table(0 if normal else 1)[3]
    k = [int(v) for v in k]
    f32 = np.float32
    out, start = [], []
    while len(out) < N:
        p0 = words.p
        u = words.next()
        i = u & 0xFF
        r = u >> 9 if normal else u >> 8
        x = f32(r) * w[i]
        if normal and (u >> 8) & 1:
            x = -x
        if r < k[i]:
            out.append(x), start.append(p0)
            continue
        if i == 0:
            if normal:
                while True:
                    a = -_log(1.0 - (words.next() >> 8) * 2.0 ** -24) / R
                    b = -_log(1.0 - (words.next() >> 8) * 2.0 ** -24)
                    if b + b > a * a:
                        break
                v = f32(R + a)
                out.append(-v if (u >> 8) & 1 else v), start.append(p0)
            else:
                out.append(f32(R - _log(1.0 - (words.next() >> 8) * 2.0 ** -24))), start.append(p0)
            continue
        U = f32((words.next() >> 8) * 2.0 ** -24)
        y = (f[i - 1] - f[i]) * U + f[i]
        if _below_exp_half_square(y, x) if normal else _below_exp(float(y), -float(x)):
            out.append(x), start.append(p0)
    return np.array(out, np.float32), np.array(start, np.uint64)


@pytest.mark.parametrize("dist", ["normal", "exp", "normalf", "expf"])
@pytest.mark.parametrize("engine,seed", [("xoshiro256pp", 2024), ("philox4x32_10", 7)])
def test_walk_with_exact_decisions_matches_the_oracle(orc, dist, engine, seed):
    normal = dist.startswith("normal")
    halves = dist.endswith("f")
    words = _Words(orc, engine, seed, halves)
    ref, ref_start = (_walk_float if halves else _walk_double)(orc, words, normal)
    got, got_start = orc.fill(orc.gen(engine, seed), dist, N, with_start=True)
    assert np.array_equal(got_start, ref_start), dist
    assert np.array_equal(got.view(np.uint32 if halves else np.uint64), ref.view(np.uint32 if halves else np.uint64)), dist


def _normal_one(words, tab):
    """One standard normal of the double walk above, with exact decisions."""
    k, w, f, R = tab
    while True:
        u = words.next()
        i = u & 0xFF
        r = (u >> 9) & (2 ** 52 - 1)
        x = float(r) * w[i]
        if (u >> 8) & 1:
            x = -x
        if r < k[i]:
            return x
        if i == 0:
            while True:
                a = -_log(1.0 - (words.next() >> 11) * 2.0 ** -53) / R
                b = -_log(1.0 - (words.next() >> 11) * 2.0 ** -53)
                if b + b > a * a:
                    break
            return -(R + a) if (u >> 8) & 1 else R + a
        U = (words.next() >> 11) * 2.0 ** -53
        y = (f[i - 1] - f[i]) * U + f[i]
        if _below_exp(y, -0.5 * (x * x)):
            return x


def _gamma_one(words, tab, alpha):
    """Marsaglia-Tsang (Sec. 3.1, Gamma), the log test decided on 40-digit
    logs; the boost for alpha < 1 draws its uniform after the accepted
    Gamma(alpha + 1)."""
    s = alpha if alpha >= 1.0 else alpha + 1.0
    d = s - 1.0 / 3.0
    with mp.workdps(40):
        c = 1.0 / float(mp.sqrt(mp.mpf(9.0 * d)))
    while True:
        x = _normal_one(words, tab)
        v = 1.0 + c * x
        if v <= 0.0:
            continue
        v = v * v * v
        U = (words.next() >> 11) * 2.0 ** -53
        x2 = x * x
        if U < 1.0 - 0.0331 * (x2 * x2) or _log(U) < 0.5 * x2 + d * ((1.0 - v) + _log(v)):
            g = d * v
            break
    if alpha >= 1.0:
        return g
    U = (words.next() >> 11) * 2.0 ** -53
    if U == 0:
        return 0.0
    with mp.workdps(40):
        return g * float(mp.exp(mp.mpf(_log(U) / alpha)))


@pytest.mark.parametrize("alpha", [0.3, 2.5])
def test_gamma_walk_with_exact_logs_matches_the_oracle(orc, alpha):
    n = 4000
    words = _Words(orc, "xoshiro256pp", 7, False)
    tab = orc.zig_table(0)
    tab = ([int(v) for v in tab[0]], tab[1], tab[2], tab[3])
    ref = np.array([_gamma_one(words, tab, alpha) for _ in range(n)])
    g = orc.gen("xoshiro256pp", 7)
    got = orc.fill(g, "gamma", n, alpha)
    assert int(g.pos) == words.p
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_beta_walk_matches_the_oracle(orc):
    """Beta (Table "continuous"): X ~ Gamma(a) drawn before Y ~ Gamma(b)."""
    n = 2000
    words = _Words(orc, "philox4x32_10", 3, False)
    tab = orc.zig_table(0)
    tab = ([int(v) for v in tab[0]], tab[1], tab[2], tab[3])
    ref = []
    for _ in range(n):
        x = _gamma_one(words, tab, 2.0)
        y = _gamma_one(words, tab, 5.0)
        ref.append(x / (x + y))
    g = orc.gen("philox4x32_10", 3)
    got = orc.fill(g, "beta", n, 2.0, 5.0)
    assert int(g.pos) == words.p
    assert np.array_equal(got.view(np.uint64), np.array(ref).view(np.uint64))
