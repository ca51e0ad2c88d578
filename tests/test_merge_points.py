"""Host checks of the chunk seams of the fill kernels.

Merge points of the gamma and t kernels
(Sec. 3.1 samplers; the seams are this library's, not the paper's).  A
chunk's merge point is found by starting the sampler at each of the first
12 word offsets of the chunk (a hypothesis that a variate starts there),
merging hypotheses that reach a variate boundary after the same word, and
stopping at the first boundary, at or after offset 11, where one chain is
left.  The true chain, which enters the chunk from the previous one, must
pass through it.  Here the rule is restated over the oracle's variate
lengths (the words one variate consumes from any start word) and checked
against the true chain of the sequential sampler, for the shapes the
library runs on these kernels: every chunk of the kernel's length (2048 or
4096 words) has a merge point, and every merge point lies on the true
chain.  The beta kernel's seams are phased merge points (hypotheses in
both phases of the X, Y alternation; _phased_point), checked the same way.

Sync points of the ziggurat normal kernel: the first position s >= G of a
chunk such that every candidate starting in [0, s) ends by s.  A true-chain
tail that starts just before the seam and overhangs it past s would leave
the previous chunk's walk mid-candidate there; the GPU fills of the same
streams are in the GPU suite."""
import numpy as np
import pytest

KE = 12   # entry offsets tried per chunk


def _one(orc, g, dist, params):
    if dist in orc.DERIVED:
        orc.fill_derived(g, dist, 1, *params)
    else:
        orc.fill(g, dist, 1, *params)


def _length_fn(orc, dist, params, seed):
    cache = {}

    def length(q):
        v = cache.get(q)
        if v is None:
            g = orc.gen("philox4x32_10", seed, pos=q)   # counter-based: any start word directly
            _one(orc, g, dist, params)
            v = cache[q] = int(g.pos) - q
        return v
    return length


def _merge_point(length, c, limit):
    nxt, alive = {}, []
    for q in range(limit):
        if q < KE:
            alive.append(q)
            nxt[q] = c + q
        idle = [e for e in alive if nxt[e] == c + q]
        if idle:
            keep = min(idle)
            alive = [e for e in alive if e == keep or e not in idle]
        if q >= KE - 1 and len(alive) == 1 and nxt[alive[0]] == c + q:
            return q
        for e in alive:
            if nxt[e] == c + q:
                nxt[e] = c + q + length(c + q)
    return -1


@pytest.mark.parametrize("dist,params,chunk", [
    ("gamma", (2.5,), 2048), ("gamma", (30.0,), 2048), ("gamma", (0.3,), 4096),
    ("beta", (2.0, 5.0), 4096), ("beta", (2.5, 3.5), 4096), ("beta", (3.0, 0.7), 4096),
    ("t", (3.0,), 4096), ("t", (100.0,), 4096),
])
def test_merge_points_exist_and_lie_on_the_true_chain(orc, dist, params, chunk):
    seed, nchunks, window = 7, 8, chunk
    length = _length_fn(orc, dist, params, seed)
    g = orc.gen("philox4x32_10", seed)
    bounds = {0}
    while max(bounds) < window * (nchunks + 1):
        _one(orc, g, dist, params)
        bounds.add(int(g.pos))
    for k in range(1, nchunks + 1):
        q = _merge_point(length, k * window, window)
        assert q >= KE - 1, (dist, params, k)
        assert k * window + q in bounds, (dist, params, k, q)


def _phased_point(len_ab, c, limit):
    """Phased merge point of the beta kernel: hypotheses (entry offset e < 12,
    phase p: 0 = X ~ Gamma(a) next, 1 = Y ~ Gamma(b) next) advance one gamma
    at a time; those at a gamma boundary after the same word in the same
    phase are one state; the point is the first word, at or after offset 11,
    after which every state left is at a gamma boundary.  Returns (q, the
    phases left) or (-1, None)."""
    pos, alive = {}, []
    for q in range(limit):
        if q < KE:
            for p in (0, 1):
                alive.append((q, p))
                pos[(q, p)] = (c + q, p)
        idle = [h for h in alive if pos[h][0] == c + q]
        for p in (0, 1):
            same = [h for h in idle if pos[h][1] == p]
            if len(same) > 1:
                drop = set(same[1:])
                alive = [h for h in alive if h not in drop]
        if q >= KE - 1 and all(pos[h][0] == c + q for h in alive):
            return q, {pos[h][1] for h in alive}
        for h in alive:
            w, p = pos[h]
            if w == c + q:
                pos[h] = (w + len_ab[p](w), 1 - p)
    return -1, None


@pytest.mark.parametrize("ab", [(2.0, 5.0), (2.0, 2.0000001), (30.0, 31.0), (0.5, 0.5000001), (3.0, 0.7)])
def test_phased_merge_points_lie_on_the_true_chain(orc, ab):
    """The beta kernel's seams: for shapes whose draws consume words alike
    (full merge points are then rare or absent) as well as for others, every
    4096-word chunk has a phased merge point, and the true chain (X, Y, X, ...
    drawn in turn by the sequential sampler) is at a gamma boundary there in
    one of the phases left."""
    seed, nchunks, window = 7, 8, 4096
    len_ab = (_length_fn(orc, "gamma", (ab[0],), seed), _length_fn(orc, "gamma", (ab[1],), seed))
    g = orc.gen("philox4x32_10", seed)
    bounds, p = {0: 0}, 0
    while max(bounds) < window * (nchunks + 1):
        orc.fill(g, "gamma", 1, ab[p])
        p = 1 - p
        bounds[int(g.pos)] = p
    for k in range(1, nchunks + 1):
        q, phases = _phased_point(len_ab, k * window, window)
        assert q >= KE - 1, (ab, k)
        assert k * window + q in bounds and bounds[k * window + q] in phases, (ab, k, q, phases)


# Normal ziggurat tails that consume 11 words (four rejected pairs), found by
# scanning the oracle's xoshiro256++ seed-2024 stream
# (tests/find_stream_cases.py): word index of the tail's first word.  A fill starting 383 words before one puts it on the
# last word of a 384-word chunk, across the seam.
LONG_TAILS = (695813604, 808170845, 1021565374)


def _candidate_len(orc, words, q, tab):
    """Words one normal candidate starting at q consumes (Sec. 3.1): 1 when
    fast, 2 for a wedge, 1 + 2k for a tail accepted at its k-th pair."""
    import mpmath as mp
    k, w, f, R = tab
    u = int(words[q])
    i, r = u & 0xFF, (u >> 9) & (2 ** 52 - 1)
    if r < int(k[i]):
        return 1
    if i:
        return 2
    j = q + 1
    while True:
        with mp.workdps(40):
            a = -float(mp.log(1 - mp.mpf((int(words[j]) >> 11) * 2.0 ** -53))) / R
            b = -float(mp.log(1 - mp.mpf((int(words[j + 1]) >> 11) * 2.0 ** -53)))
        j += 2
        if b + b > a * a:
            return j - q


def _sync_point(orc, words, c, g, s_win, tab):
    reach = 0
    for q in range(g + s_win):
        if q >= g and reach <= q:
            return q
        reach = max(reach, q + _candidate_len(orc, words, c + q, tab))
    return -1


@pytest.mark.parametrize("w", LONG_TAILS)
def test_normal_sync_points_clear_an_overhanging_tail(orc, w):
    """With sync points from 16 on, the chunk after the seam starts its
    chain after the 11-word tail has ended; from 8 on (the earlier rule) it
    would start inside it."""
    chunk, pos = 384, w - 383
    words = orc.next_words(orc.gen("xoshiro256pp", 2024, pos=pos), 1200)
    tab = orc.zig_table(0)
    assert _candidate_len(orc, words, chunk - 1, tab) == 11
    _, start = orc.fill(orc.gen("xoshiro256pp", 2024, pos=pos), "normal", 600, with_start=True)
    assert w in set(int(x) for x in start)   # on the true chain of a fill from pos
    tail_end = chunk - 1 + 11 - chunk        # relative to the next chunk
    assert _sync_point(orc, words, chunk, 16, 16, tab) >= tail_end
    assert _sync_point(orc, words, chunk, 8, 24, tab) < tail_end
