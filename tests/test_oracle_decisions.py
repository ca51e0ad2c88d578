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

mp.mp.dps = 40
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
    return float(mp.log(mp.mpf(x)))   # rounded to nearest from 40 digits


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
        if mp.mpf(y) < mp.exp(mp.mpf(t)):
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
        xm = mp.mpf(float(x))
        t = -xm * xm / 2 if normal else -xm
        if mp.mpf(float(y)) < mp.exp(t):
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
