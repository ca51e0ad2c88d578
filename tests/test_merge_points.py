"""Host check of the merge-point seams of the gamma, beta and t kernels
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
chain."""
import numpy as np
import pytest

KE = 12   # entry offsets tried per chunk


def _length_fn(orc, dist, params, seed):
    cache = {}

    def length(q):
        v = cache.get(q)
        if v is None:
            g = orc.gen("philox4x32_10", seed, pos=q)   # counter-based: any start word directly
            orc.fill(g, dist, 1, *params)
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
])
def test_merge_points_exist_and_lie_on_the_true_chain(orc, dist, params, chunk):
    seed, nchunks, window = 7, 8, chunk
    length = _length_fn(orc, dist, params, seed)
    g = orc.gen("philox4x32_10", seed)
    bounds = {0}
    while max(bounds) < window * (nchunks + 1):
        orc.fill(g, dist, 1, *params)
        bounds.add(int(g.pos))
    for k in range(1, nchunks + 1):
        q = _merge_point(length, k * window, window)
        assert q >= KE - 1, (dist, params, k)
        assert k * window + q in bounds, (dist, params, k, q)
