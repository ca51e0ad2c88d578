"""ctypes front-end of the serial C oracle.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, serial CPU
implementation of the bulk-fill hot path of Randompack (arXiv 2605.05099):
engines (Sec. 2.2), seeding and jumps (Sec. 2.3, Sec. 4.4), U(0,1) and the
bounded integers (Sec. 3.1-3.2), ziggurat normal/exponential (Sec. 3.1),
Marsaglia--Tsang gamma and beta (Sec. 3.1), pathwise gradients and the MVN
transform.  Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the CUDA library never calls it.

Parity status per function (see the tests under tests/test_oracle_*.py):
every function is pinned against something other than itself (NumPy
black-box engines and SeedSequence, closed forms, brute force, jump
identities, mpmath quadrature, SciPy finite differences, statistical tests).
One exception: the constants of the xoshiro256** scrambler (5, 7, 9) come
from the engine's published definition with no independent vectors here,
so for them the parity is unpinned; which state word it scrambles, the
order of its steps and the transition under it are pinned.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

XOSHIRO256PP, PCG64DXSM, PHILOX4X32_10, PHILOX4X64_10, XOSHIRO256SS = 1, 2, 3, 4, 5
ENGINES = {"xoshiro256pp": XOSHIRO256PP, "pcg64dxsm": PCG64DXSM, "philox4x32_10": PHILOX4X32_10,
           "philox4x64_10": PHILOX4X64_10, "xoshiro256ss": XOSHIRO256SS}


def build(force=False):
    """Compile liboracle.so with gcc (-O2, no FP contraction, no fast-math)."""
    src = [os.path.join(_HERE, "rp_oracle.c")]
    deps = src + [os.path.join(_HERE, f) for f in ("rp_oracle.h", "ziggurat_tables.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + src + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class Gen(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int), ("s", ctypes.c_uint64 * 4), ("pos", ctypes.c_uint64),
                ("blk_idx", ctypes.c_uint64), ("blk_valid", ctypes.c_int),
                ("blk", ctypes.c_uint64 * 4)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u64, i32, dbl, sz = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        sig = {
            "or_seedseq_generate": (None, [vp, i32, vp, i32]),
            "or_seedseq_entropy": (i32, [u64, i32, u64, vp]),
            "or_gen_seed": (i32, [P(Gen), i32, u64, i32, u64]),
            "or_gen_set": (None, [P(Gen), i32, vp]),
            "or_next": (u64, [P(Gen)]),
            "or_jump": (None, [P(Gen), u64, u64]),
            "or_seek": (None, [P(Gen), u64]),
            "or_xoshiro_jump_poly": (None, [vp, vp, i32]),
            "or_xoshiro_jump_matrix": (None, [vp, vp, i32]),
            "or_xoshiro_charpoly": (None, [vp]),
            "or_pcg_advance": (None, [vp, u64, u64]),
            "or_philox4x32_10": (None, [vp, vp, vp]),
            "or_philox4x64_10": (None, [vp, vp, vp]),
            "or_fill_uniform52": (None, [P(Gen), sz, vp]),
            "or_cr_exp": (dbl, [dbl]),
            "or_cr_log": (dbl, [dbl]),
            "or_cr_ambiguous": (u64, []),
            "or_cr_reset": (None, []),
            "or_fill_u64": (None, [P(Gen), sz, vp]),
            "or_fill_uniform": (None, [P(Gen), sz, vp]),
            "or_fill_bounded": (None, [P(Gen), sz, u64, vp, vp]),
            "or_fill_normal": (None, [P(Gen), sz, vp, vp]),
            "or_fill_exp": (None, [P(Gen), sz, vp, vp]),
            "or_fill_uniformf": (None, [P(Gen), sz, vp]),
            "or_fill_normalf": (None, [P(Gen), sz, vp, vp]),
            "or_fill_expf": (None, [P(Gen), sz, vp, vp]),
            "or_zig_table_f": (i32, [i32, i32, P(ctypes.c_uint32), P(ctypes.c_float), P(ctypes.c_float)]),
            "or_fill_gamma": (i32, [P(Gen), sz, dbl, vp, vp]),
            "or_fill_beta": (i32, [P(Gen), sz, dbl, dbl, vp, vp]),
            "or_fill_derived": (i32, [P(Gen), i32, sz, vp, vp, vp]),
            "or_cr_pow": (dbl, [dbl, dbl]),
            "or_zig_normal_x": (dbl, [u64]),
            "or_zig_table": (i32, [i32, i32, P(u64), P(dbl), P(dbl)]),
            "or_zig_R": (dbl, [i32]),
            "or_zig_counts": (None, [vp]),
            "or_digamma": (dbl, [dbl]),
            "or_gamma_dzda": (dbl, [dbl, dbl]),
            "or_beta_dzdab": (None, [dbl, dbl, dbl, P(dbl), P(dbl)]),
            "or_beta_dzdab_composed": (None, [dbl, dbl, dbl, dbl, P(dbl), P(dbl)]),
            "or_mvn_apply": (None, [i32, sz, vp, vp, vp, vp]),
            "or_mvn_grads": (None, [i32, sz, vp, vp, vp, vp]),
            "or_substream": (None, [P(Gen), i32, u64, u64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# ---------------------------------------------------------------- generators
NO_STREAM = None


def gen(engine, seed, stream=None, pos=0):
    """Seeded generator at word position `pos`; stream = spawn key or None."""
    g = Gen()
    eng = ENGINES[engine] if isinstance(engine, str) else engine
    rc = lib().or_gen_seed(ctypes.byref(g), eng, seed, 0 if stream is None else 1,
                           0 if stream is None else stream)
    if rc != 0:
        raise ValueError("all-zero seeded state")
    if pos:
        lib().or_seek(ctypes.byref(g), pos)
    return g


def substream(engine, base_seed, s):
    g = Gen()
    eng = ENGINES[engine] if isinstance(engine, str) else engine
    lib().or_substream(ctypes.byref(g), eng, base_seed, s)
    return g


def jump(g, n):
    """Advance a generator by n words (or_jump)."""
    lib().or_jump(ctypes.byref(g), (n >> 64) & (2**64 - 1), n & (2**64 - 1))
    return g


def state_words(g):
    return [int(x) for x in g.s]


def next_words(g, n):
    out = np.empty(n, np.uint64)
    lib().or_fill_u64(ctypes.byref(g), n, _ptr(out))
    return out


def seedseq_generate(entropy_words, n_out):
    ent = np.asarray(entropy_words, np.uint32)
    out = np.empty(n_out, np.uint32)
    lib().or_seedseq_generate(_ptr(ent), len(ent), _ptr(out), n_out)
    return out


def seedseq_entropy(seed, key=None):
    ent = np.zeros(8, np.uint32)
    n = lib().or_seedseq_entropy(seed, 0 if key is None else 1, 0 if key is None else key, _ptr(ent))
    return ent[:n]


def xoshiro_jump(state, n, method="poly"):
    s = np.array(state, np.uint64)
    limbs = []
    while True:
        limbs.append(n & (2 ** 64 - 1))
        n >>= 64
        if n == 0:
            break
    nl = np.array(limbs, np.uint64)
    f = lib().or_xoshiro_jump_poly if method == "poly" else lib().or_xoshiro_jump_matrix
    f(_ptr(s), _ptr(nl), len(limbs))
    return [int(x) for x in s]


def xoshiro_charpoly():
    p = np.zeros(5, np.uint64)
    lib().or_xoshiro_charpoly(_ptr(p))
    return sum(int(w) << (64 * i) for i, w in enumerate(p))


def pcg_advance(state4, delta):
    s = np.array(state4, np.uint64)
    lib().or_pcg_advance(_ptr(s), (delta >> 64) & (2 ** 64 - 1), delta & (2 ** 64 - 1))
    return [int(x) for x in s]


def philox4x64(ctr4, key2):
    c = np.array(ctr4, np.uint64)
    k = np.array(key2, np.uint64)
    o = np.empty(4, np.uint64)
    lib().or_philox4x64_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


def philox(ctr4, key2):
    c = np.array(ctr4, np.uint32)
    k = np.array(key2, np.uint32)
    o = np.empty(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


# ---------------------------------------------------------------- fills
def fill(g, dist, n, *params, with_start=False):
    """Run one oracle fill on generator g (advances g).  Returns out (and
    start positions when with_start)."""
    L = lib()
    gp = ctypes.byref(g)
    start = np.empty(n, np.uint64) if with_start else None
    if dist == "u64":
        out = np.empty(n, np.uint64)
        L.or_fill_u64(gp, n, _ptr(out))
        if with_start:
            start[:] = np.arange(n, dtype=np.uint64) + np.uint64(g.pos - n)
    elif dist == "uniform":
        out = np.empty(n, np.float64)
        L.or_fill_uniform(gp, n, _ptr(out))
        if with_start:
            start[:] = np.arange(n, dtype=np.uint64) + np.uint64(g.pos - n)
    elif dist == "uniform52":
        out = np.empty(n, np.float64)
        L.or_fill_uniform52(gp, n, _ptr(out))
        if with_start:
            start[:] = np.arange(n, dtype=np.uint64) + np.uint64(g.pos - n)
    elif dist == "bounded":
        out = np.empty(n, np.uint64)
        L.or_fill_bounded(gp, n, params[0], _ptr(out), _ptr(start))
    elif dist == "normal":
        out = np.empty(n, np.float64)
        L.or_fill_normal(gp, n, _ptr(out), _ptr(start))
    elif dist == "exp":
        out = np.empty(n, np.float64)
        L.or_fill_exp(gp, n, _ptr(out), _ptr(start))
    elif dist == "uniformf":
        out = np.empty(n, np.float32)
        L.or_fill_uniformf(gp, n, _ptr(out))
        if with_start:
            raise ValueError("uniformf has one 32-bit word per output: no start list")
    elif dist == "normalf":
        out = np.empty(n, np.float32)
        L.or_fill_normalf(gp, n, _ptr(out), _ptr(start))
    elif dist == "expf":
        out = np.empty(n, np.float32)
        L.or_fill_expf(gp, n, _ptr(out), _ptr(start))
    elif dist == "gamma":
        out = np.empty(n, np.float64)
        if L.or_fill_gamma(gp, n, float(params[0]), _ptr(out), _ptr(start)) != 0:
            raise ValueError("alpha must be > 0")
    elif dist == "beta":
        out = np.empty(n, np.float64)
        if L.or_fill_beta(gp, n, float(params[0]), float(params[1]), _ptr(out), _ptr(start)) != 0:
            raise ValueError("a, b must be > 0")
    else:
        raise ValueError(dist)
    return (out, start) if with_start else out


# derived distributions (Table "continuous"): name -> (kind, parameter names)
DERIVED = {"unif": (1, ("a", "b")), "normal_ms": (2, ("mu", "sigma")), "lognormal": (3, ("mu", "sigma")),
           "exp_scale": (4, ("beta",)), "gamma_scale": (5, ("alpha", "theta")), "chi2": (6, ("nu",)),
           "gumbel": (7, ("mu", "beta")), "pareto": (8, ("x_m", "alpha")), "weibull": (9, ("k", "lambda")),
           "gpd": (10, ("mu", "sigma", "xi")), "f": (11, ("nu1", "nu2")), "skew_normal": (12, ("mu", "sigma", "alpha")),
           "t": (13, ("nu",))}


def fill_derived(g, name, n, *params, with_start=False):
    """One derived-distribution fill on generator g (advances g)."""
    kind, names = DERIVED[name]
    if len(params) != len(names):
        raise ValueError(f"{name} takes {names}")
    p = np.zeros(4, np.float64)
    p[: len(params)] = params
    out = np.empty(n, np.float64)
    start = np.empty(n, np.uint64) if with_start else None
    if lib().or_fill_derived(ctypes.byref(g), kind, n, _ptr(p), _ptr(out), _ptr(start)) != 0:
        raise ValueError(f"bad parameters for {name}")
    return (out, start) if with_start else out


def cr_pow(x, y):
    return lib().or_cr_pow(float(x), float(y))


def zig_counts():
    c = np.zeros(4, np.uint64)
    lib().or_zig_counts(_ptr(c))
    return dict(fast=int(c[0]), wedge=int(c[1]), reject=int(c[2]), tail=int(c[3]))


def zig_table_f(which):
    """Float tables of the f variants, derived from the double ones:
    which 0 normal, 1 exponential -> (k uint32[256], w, f float32[256])"""
    k = np.empty(256, np.uint32)
    w = np.empty(256, np.float32)
    f = np.empty(256, np.float32)
    kk, ww, ff = ctypes.c_uint32(), ctypes.c_float(), ctypes.c_float()
    for i in range(256):
        lib().or_zig_table_f(which, i, ctypes.byref(kk), ctypes.byref(ww), ctypes.byref(ff))
        k[i], w[i], f[i] = kk.value, ww.value, ff.value
    return k, w, f


def zig_table(which):
    """which: 0 normal, 1 exponential -> (k uint64[256], w, f float64[256], R)"""
    k = np.empty(256, np.uint64)
    w = np.empty(256)
    f = np.empty(256)
    kk, ww, ff = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    for i in range(256):
        lib().or_zig_table(which, i, ctypes.byref(kk), ctypes.byref(ww), ctypes.byref(ff))
        k[i], w[i], f[i] = kk.value, ww.value, ff.value
    return k, w, f, lib().or_zig_R(which)


def cr_exp(x):
    return lib().or_cr_exp(float(x))


def cr_log(x):
    return lib().or_cr_log(float(x))


def cr_ambiguous():
    return int(lib().or_cr_ambiguous())


def digamma(x):
    return lib().or_digamma(float(x))


def gamma_dzda(z, alpha):
    return lib().or_gamma_dzda(float(z), float(alpha))


def beta_dzdab(z, a, b):
    da, db = ctypes.c_double(), ctypes.c_double()
    lib().or_beta_dzdab(float(z), float(a), float(b), ctypes.byref(da), ctypes.byref(db))
    return da.value, db.value


def beta_dzdab_composed(x, y, a, b):
    da, db = ctypes.c_double(), ctypes.c_double()
    lib().or_beta_dzdab_composed(float(x), float(y), float(a), float(b), ctypes.byref(da), ctypes.byref(db))
    return da.value, db.value


def beta_pairs(g, n, a, b):
    """The gamma pairs (X, Y) that the beta fill draws: X ~ Gamma(a) before
    Y ~ Gamma(b), n times, from generator g."""
    xy = np.empty((n, 2))
    for j in range(n):
        xy[j, 0] = fill(g, "gamma", 1, a)[0]
        xy[j, 1] = fill(g, "gamma", 1, b)[0]
    return xy


def mvn_apply(mu, L, Z):
    d = len(mu)
    Z = np.ascontiguousarray(Z, np.float64)
    n = Z.shape[0]
    X = np.empty((n, d))
    lib().or_mvn_apply(d, n, _ptr(np.ascontiguousarray(mu, np.float64)),
                       _ptr(np.ascontiguousarray(L, np.float64)), _ptr(Z), _ptr(X))
    return X


def mvn_grads(G, Z):
    G = np.ascontiguousarray(G, np.float64)
    Z = np.ascontiguousarray(Z, np.float64)
    n, d = G.shape
    gmu = np.empty(d)
    gL = np.empty((d, d))
    lib().or_mvn_grads(d, n, _ptr(G), _ptr(Z), _ptr(gmu), _ptr(gL))
    return gmu, gL
