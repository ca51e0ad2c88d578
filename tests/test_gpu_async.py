"""Asynchronous fills (the boundary's *pos contract): one-word fills return
without waiting; the sampled fills, given a position in pinned host memory,
return without waiting and write the end position there once the stream
reaches it.  Values and positions must equal the synchronous calls bit for
bit; fills chained through one pinned word and fills on two streams must
stay correct; device failures must show as an all-ones position and be
reported by rp_async_status (Sec. 2.1: errors are returned)."""
import time

import numpy as np
import pytest
import torch

import paper_2605_05099_gb300 as rp
from gpu_util import DTYPE

pytestmark = pytest.mark.gpu

FILLS = {
    "normal": lambda e, s, p, o, cs: rp.rp_fill_normal(e, s, rp.NO_STREAM, p, o, cs),
    "exp": lambda e, s, p, o, cs: rp.rp_fill_exp(e, s, rp.NO_STREAM, p, o, cs),
    "gamma": lambda e, s, p, o, cs: rp.rp_fill_gamma(e, s, rp.NO_STREAM, p, 2.5, o, cs),
    "beta": lambda e, s, p, o, cs: rp.rp_fill_beta(e, s, rp.NO_STREAM, p, 2.0, 5.0, o, cs),
    "bounded6": lambda e, s, p, o, cs: rp.rp_fill_bounded(e, s, rp.NO_STREAM, p, 6, o, cs),
    "bounded_half": lambda e, s, p, o, cs: rp.rp_fill_bounded(e, s, rp.NO_STREAM, p, (1 << 63) + 1, o, cs),
    "u64": lambda e, s, p, o, cs: rp.rp_fill_u64(e, s, rp.NO_STREAM, p, o, cs),
    "uniform": lambda e, s, p, o, cs: rp.rp_fill_uniform(e, s, rp.NO_STREAM, p, o, cs),
}
KIND = {"bounded6": "bounded", "bounded_half": "bounded"}


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rp.rp_debug_faults("clear")
    yield
    rp.rp_debug_faults("clear")


def _pinned(v):
    t = torch.empty(1, dtype=torch.int64).pin_memory()
    t[0] = v
    return t


def _bits(t):
    if t.dtype == torch.uint64:
        return t.view(torch.int64).cpu().numpy()
    return t.cpu().numpy().view(np.int64)


def _new(dist, n):
    return torch.empty(n, dtype=DTYPE[KIND.get(dist, dist)], device="cuda")


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10"])
@pytest.mark.parametrize("dist", list(FILLS))
def test_async_equals_sync(engine, dist):
    n, start = 100_003, 5
    ref = _new(dist, n)
    pos_ref = FILLS[dist](engine, 77, start, ref, None)
    got = _new(dist, n)
    pp = _pinned(start)
    assert FILLS[dist](engine, 77, pp, got, None) is None
    torch.cuda.synchronize()
    rp.rp_async_status()
    assert int(pp[0]) == pos_ref
    assert np.array_equal(_bits(got), _bits(ref))


def test_chain_through_one_pinned_word():
    """Three sampled fills and a one-word fill chained through one pinned
    position, with no synchronisation between them, equal the synchronous
    chain."""
    n = 50_000
    seq = ["normal", "gamma", "u64", "exp"]
    pos, refs = 0, []
    for d in seq:
        r = _new(d, n)
        pos = FILLS[d]("xoshiro256pp", 3, pos, r, None)
        refs.append(r)
    pp = _pinned(0)
    outs = []
    for d in seq:
        o = _new(d, n)
        FILLS[d]("xoshiro256pp", 3, pp, o, None)
        outs.append(o)
    torch.cuda.synchronize()
    rp.rp_async_status()
    assert int(pp[0]) == pos
    for o, r in zip(outs, refs):
        assert np.array_equal(_bits(o), _bits(r))


def test_two_streams_share_the_scratch():
    """Sampled fills issued alternately on two streams (each with its own
    pinned position) are ordered around the shared scratch on the device."""
    n = 200_000
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    want = []
    for k in range(4):
        a, b = _new("normal", n), _new("gamma", n)
        pa = FILLS["normal"]("philox4x32_10", 10 + k, 0, a, None)
        pb = FILLS["gamma"]("pcg64dxsm", 20 + k, 0, b, None)
        want.append((a, pa, b, pb))
    got = []
    for k in range(4):
        a, b = _new("normal", n), _new("gamma", n)
        qa, qb = _pinned(0), _pinned(0)
        FILLS["normal"]("philox4x32_10", 10 + k, qa, a, s1)
        FILLS["gamma"]("pcg64dxsm", 20 + k, qb, b, s2)
        got.append((a, qa, b, qb))
    torch.cuda.synchronize()
    rp.rp_async_status()
    for (a, pa, b, pb), (a2, qa, b2, qb) in zip(want, got):
        assert int(qa[0]) == pa and int(qb[0]) == pb
        assert np.array_equal(_bits(a2), _bits(a)) and np.array_equal(_bits(b2), _bits(b))


@pytest.mark.parametrize("dist,pinned", [("u64", False), ("uniform", False), ("normal", True), ("gamma", True)])
def test_calls_return_before_the_stream_reaches_them(dist, pinned):
    """With the stream held by a ~0.2 s spin kernel, the call returns long
    before the spin ends (one-word fills always; sampled fills with a
    pinned position)."""
    n = 1 << 20
    out = _new(dist, n)
    FILLS[dist]("xoshiro256pp", 1, 0, out, None)      # tables and scratch set up
    torch.cuda.synchronize()
    torch.cuda._sleep(400_000_000)                     # 0.2 s at 2 GHz
    t0 = time.perf_counter()
    p = _pinned(0) if pinned else 0
    FILLS[dist]("xoshiro256pp", 1, p, out, None)
    dt = time.perf_counter() - t0
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    assert dt < 0.05 and wall > 0.1, (dt, wall)


def test_failures_are_reported_after_the_sync():
    """An asynchronous fill that runs out of its planned tiles, and one whose
    look-back waits run out, leave an all-ones position and an error that
    rp_async_status reports once; the next fill is correct again."""
    n = 1 << 20
    out = _new("normal", n)
    rp.rp_debug_faults("tile_cap", 2)
    pp = _pinned(0)
    FILLS["normal"]("xoshiro256pp", 9, pp, out, None)
    torch.cuda.synchronize()
    assert int(pp[0]) == -1
    with pytest.raises(rp.RPError) as ei:
        rp.rp_async_status()
    assert ei.value.code == -7 and "planned tiles" in str(ei.value)
    rp.rp_async_status()                               # cleared
    rp.rp_debug_faults("clear")
    rp.rp_debug_faults("spin_max", 2000)
    rp.rp_debug_faults("stall_tile", 5)
    pp = _pinned(0)
    FILLS["exp"]("philox4x32_10", 9, pp, _new("exp", 1 << 22), None)
    torch.cuda.synchronize()
    assert int(pp[0]) == -1
    with pytest.raises(rp.RPError) as ei:
        rp.rp_async_status()
    assert ei.value.code == -5
    rp.rp_debug_faults("clear")
    ref = _new("normal", n)
    pos = FILLS["normal"]("xoshiro256pp", 9, 0, ref, None)
    pp = _pinned(0)
    FILLS["normal"]("xoshiro256pp", 9, pp, out, None)
    torch.cuda.synchronize()
    rp.rp_async_status()
    assert int(pp[0]) == pos and np.array_equal(_bits(out), _bits(ref))


@pytest.mark.parametrize("dist,params", [("normal", ()), ("bounded", (6,)), ("gamma", (2.5,)), ("u64", ())])
@pytest.mark.parametrize("pinned", [True, False])
def test_fill_to_host(dist, params, pinned):
    """rp_fill_to_host: the same values and position as the device fill, in
    pinned (asynchronous) and pageable host memory; consecutive calls
    alternate staging slots, so three calls in a row must all land."""
    n = 300_001
    kw = {"p0": params[0]} if dist == "gamma" else ({"m": params[0]} if dist == "bounded" else {})
    refs, outs, poss = [], [], []
    pos = 0
    for k in range(3):
        r = _new(dist if dist != "bounded" else "bounded6", n)
        pos = FILLS[{"normal": "normal", "bounded": "bounded6", "gamma": "gamma", "u64": "u64"}[dist]](
            "philox4x32_10", 77, pos, r, None)
        refs.append(r)
    p = 0
    for k in range(3):
        h = torch.empty(n, dtype=torch.int64)
        if pinned:
            h = h.pin_memory()
        p = rp.rp_fill_to_host("philox4x32_10", 77, rp.NO_STREAM, p, dist, h, **kw)
        outs.append(h)
    torch.cuda.synchronize()
    rp.rp_async_status(None)
    assert p == pos
    for h, r in zip(outs, refs):
        assert np.array_equal(h.numpy(), _bits(r))


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10"])
def test_one_word_fills_replay_from_a_cuda_graph(engine):
    """One-word fills issue no host wait and no stream-ordered library call
    besides their kernel, so once their tables are in place (one call with
    the same engine and size) they can be captured into a CUDA graph: the
    replay writes what the calls write."""
    n = (1 << 18) + 77
    w = torch.empty(n, dtype=torch.uint64, device="cuda")
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    f = torch.empty(2 * n, dtype=torch.float32, device="cuda")

    def fills(cs):
        p = rp.rp_fill_u64(engine, 41, rp.NO_STREAM, 3, w, cs)
        p = rp.rp_fill_uniform(engine, 41, rp.NO_STREAM, p, u, cs)
        return rp.rp_fill_uniformf(engine, 41, rp.NO_STREAM, p, f, cs)

    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        end = fills(cap)
    torch.cuda.synchronize()
    ref = (_bits(w).copy(), _bits(u).copy(), f.cpu().numpy().view(np.int32).copy())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
        assert fills(cap) == end
    for t in (w, u, f):
        t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(_bits(w), ref[0]) and np.array_equal(_bits(u), ref[1])
    assert np.array_equal(f.cpu().numpy().view(np.int32), ref[2])
