"""Host model of the second pass of the bounded fill with frequent
rejections (rej_tile in csrc/rp_rej.cuh): a warp holds 32 parked runs of
cnt[r] <= C words, run r starting at output off[r] (an exclusive scan over
the warp's lanes plus the warp's base); the warp loads run r + 1 while it
stores run r, Q = C / 32 rows of 32 lanes per run, each store clipped to the
`lim` outputs left in the fill.  Every output below lim must receive exactly
the parked word of its run and rank, and no store may reach lim or beyond.
A check of the kernel's method on the host, not of the oracle."""
import numpy as np
import pytest

C = 256


def model(cnt, base, lim):
    Q = C // 32
    off = base + np.concatenate([[0], np.cumsum(cnt)[:-1]])
    park = [[(r, k) for k in range(cnt[r])] + [None] * (C - cnt[r]) for r in range(32)]
    out = {}

    def load(r, c):
        return [[park[r][q * 32 + lane] if q * 32 + lane < c else 0 for lane in range(32)] for q in range(Q)]

    o = int(off[0])
    c = min(int(cnt[0]), lim - o)
    v = load(0, c)
    for r in range(32):
        o2 = c2 = 0
        w = None
        if r + 1 < 32:
            o2 = int(off[r + 1])
            c2 = min(int(cnt[r + 1]), lim - o2)
            w = load(r + 1, c2)
        for q in range(Q):
            for lane in range(32):
                i = q * 32 + lane
                if i < c:
                    assert o + i < lim
                    assert o + i not in out
                    out[o + i] = v[q][lane]
        v, o, c = w, o2, c2
    return out, off


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("clip", [False, True])
def test_runs_land_once_in_order(seed, clip):
    rng = np.random.default_rng(seed)
    cnt = rng.binomial(C, 0.5, size=32)
    if seed % 3 == 0:
        cnt[rng.integers(0, 32, 4)] = 0           # empty runs
    if seed % 4 == 1:
        cnt[rng.integers(0, 32, 2)] = C           # full runs
    base = int(rng.integers(0, 1000))
    total = int(cnt.sum())
    lim = base + (int(rng.integers(0, total + 1)) if clip else total)
    out, off = model(cnt, base, lim)
    assert sorted(out) == list(range(base, lim))
    for r in range(32):
        for k in range(cnt[r]):
            p = int(off[r]) + k
            if p < lim:
                assert out[p] == (r, k)
