"""Helpers shared by the GPU tests: run a fill through the C ABI and the same
fill through the oracle."""
import numpy as np
import torch

import oracle
import paper_2605_05099_gb300 as rp

DTYPE = {"u64": torch.uint64, "uniform": torch.float64, "uniform52": torch.float64, "bounded": torch.uint64, "normal": torch.float64,
         "exp": torch.float64, "gamma": torch.float64, "beta": torch.float64}


def gpu_fill(dist, engine, seed, stream, pos, n, params=()):
    out = torch.empty(n, dtype=DTYPE[dist], device="cuda")
    s = rp.NO_STREAM if stream is None else stream
    if dist == "u64":
        newpos = rp.rp_fill_u64(engine, seed, s, pos, out)
    elif dist == "uniform":
        newpos = rp.rp_fill_uniform(engine, seed, s, pos, out)
    elif dist == "uniform52":
        newpos = rp.rp_fill_uniform52(engine, seed, s, pos, out)
    elif dist == "bounded":
        newpos = rp.rp_fill_bounded(engine, seed, s, pos, params[0], out)
    elif dist == "normal":
        newpos = rp.rp_fill_normal(engine, seed, s, pos, out)
    elif dist == "exp":
        newpos = rp.rp_fill_exp(engine, seed, s, pos, out)
    elif dist == "gamma":
        newpos = rp.rp_fill_gamma(engine, seed, s, pos, params[0], out)
    elif dist == "beta":
        newpos = rp.rp_fill_beta(engine, seed, s, pos, params[0], params[1], out)
    torch.cuda.synchronize()
    if out.dtype == torch.uint64:
        host = out.view(torch.int64).cpu().numpy().view(np.uint64)
    else:
        host = out.cpu().numpy()
    return host, newpos


def oracle_fill(dist, engine, seed, stream, pos, n, params=(), with_start=False):
    g = oracle.gen(engine, seed, stream, pos=pos)
    if with_start:
        out, start = oracle.fill(g, dist, n, *params, with_start=True)
        return out, int(g.pos), start
    out = oracle.fill(g, dist, n, *params)
    return out, int(g.pos)


# Bars for outputs built from gamma variates that went through the boost
# for shapes below 1 (a libm exp; each such gamma is within 2 ulp, the bar
# for transcendental outputs).  With X^ = X (1 + a), |a| <= 2 ulp(X)/X <=
# 2^-51, likewise b for Y, and unit roundoff 2^-53 per IEEE operation, the
# first-order relative error of each formula, over ulp(z) > z 2^-53, gives:
#   beta   X/(X+Y):              (1-z)(|a|+|b|) + 2 roundings -> < 8 + 2 = 10 ulp
#   F      (X/n1)/(Y/n2):        |a| + |b| + 3 roundings      -> < 8 + 3 = 11 ulp
#   Gamma(alpha, theta)  X theta: |a| + 1 rounding            -> < 4 + 1 = 5 ulp
#   t      Z / sqrt(2 G / nu):   (|a| + 1 rounding)/2 under the root, then the
#                                root and the quotient: 2 roundings -> < 2.5 + 2 < 5 ulp
BOOST_ULP = {"beta": 10, "f": 11, "gamma_scale": 5, "t": 5}


def ulp_diff(a, b):
    """distance in units in the last place between doubles of the same sign"""
    ia = np.asarray(a, np.float64).view(np.int64).astype(object)
    ib = np.asarray(b, np.float64).view(np.int64).astype(object)
    return abs(int(ia) - int(ib))


def tail_output(dist, engine, seed, stream, start_pos):
    """True when the candidate that produced an output began in the
    ziggurat base strip beyond the fast-accept threshold (the tail)."""
    if dist not in ("normal", "exp"):
        return False
    g = oracle.gen(engine, seed, stream, pos=int(start_pos))
    u = int(oracle.next_words(g, 1)[0])
    which = 0 if dist == "normal" else 1
    k0 = int(oracle.zig_table(which)[0][0])
    r = (u >> 9) & (2 ** 52 - 1) if dist == "normal" else (u >> 8) & (2 ** 53 - 1)
    return (u & 0xFF) == 0 and r >= k0


def assert_parity(dist, engine, seed, stream, pos, n, params=(), max_tail_ulp=2):
    """GPU fill vs oracle: identical consumed words and accept sequence;
    outputs bit-identical except tail outputs of the ziggurat samplers, whose
    values go through log and must be within max_tail_ulp."""
    g, gpos = gpu_fill(dist, engine, seed, stream, pos, n, params)
    o, opos, start = oracle_fill(dist, engine, seed, stream, pos, n, params, with_start=True)
    assert gpos == opos, (dist, engine, n, gpos, opos)
    ug, uo = g.view(np.uint64), o.view(np.uint64)
    bad = np.nonzero(ug != uo)[0]
    assert len(bad) <= max(8, n // 1000), (dist, engine, n, len(bad))
    for j in bad:
        assert tail_output(dist, engine, seed, stream, start[j]), (dist, engine, n, int(j), g[j], o[j])
        assert ulp_diff(g[j], o[j]) <= max_tail_ulp, (dist, engine, int(j), g[j], o[j])
    return len(bad)


def same_bits(a, b):
    return a.dtype.itemsize == b.dtype.itemsize and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def first_mismatch(a, b):
    ua, ub = a.view(np.uint64), b.view(np.uint64)
    idx = np.nonzero(ua != ub)[0]
    return int(idx[0]) if len(idx) else -1
