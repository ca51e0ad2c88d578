"""Helpers shared by the GPU tests: run a fill through the C ABI and the same
fill through the oracle."""
import numpy as np
import torch

import oracle
import paper_2605_05099_gb300 as rp

DTYPE = {"u64": torch.uint64, "uniform": torch.float64, "bounded": torch.uint64, "normal": torch.float64,
         "exp": torch.float64, "gamma": torch.float64, "beta": torch.float64}


def gpu_fill(dist, engine, seed, stream, pos, n, params=()):
    out = torch.empty(n, dtype=DTYPE[dist], device="cuda")
    s = rp.NO_STREAM if stream is None else stream
    if dist == "u64":
        newpos = rp.rp_fill_u64(engine, seed, s, pos, out)
    elif dist == "uniform":
        newpos = rp.rp_fill_uniform(engine, seed, s, pos, out)
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


def oracle_fill(dist, engine, seed, stream, pos, n, params=()):
    g = oracle.gen(engine, seed, stream, pos=pos)
    out = oracle.fill(g, dist, n, *params)
    return out, int(g.pos)


def same_bits(a, b):
    return a.dtype.itemsize == b.dtype.itemsize and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def first_mismatch(a, b):
    ua, ub = a.view(np.uint64), b.view(np.uint64)
    idx = np.nonzero(ua != ub)[0]
    return int(idx[0]) if len(idx) else -1
