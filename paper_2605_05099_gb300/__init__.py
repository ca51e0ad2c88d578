"""Python binding of librp, the GB300 bulk-fill library (C ABI in include/rp.h).

Argument marshalling only: every fill runs in the CUDA kernels of librp.so.
PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback; a missing or unloadable library raises immediately.

    import torch, paper_2605_05099_gb300 as rp
    x = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    pos = rp.rp_fill_normal(rp.XOSHIRO256PP, 12345, rp.NO_STREAM, 0, x)
"""
import ctypes
import os

import torch

XOSHIRO256PP, PCG64DXSM, PHILOX4X32_10, PHILOX4X64_10, XOSHIRO256SS = 1, 2, 3, 4, 5
DISTS = {"u64": 0, "uniform": 1, "bounded": 2, "normal": 3, "exp": 4, "gamma": 5, "beta": 6, "uniform52": 7}
ENGINES = {"xoshiro256pp": XOSHIRO256PP, "pcg64dxsm": PCG64DXSM, "philox4x32_10": PHILOX4X32_10,
           "philox4x64_10": PHILOX4X64_10, "xoshiro256ss": XOSHIRO256SS}
NO_STREAM = (1 << 64) - 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librp.so")

STATUS = {0: "RP_OK", -1: "RP_ERR_NULL", -2: "RP_ERR_PARAM", -3: "RP_ERR_ENGINE", -4: "RP_ERR_CUDA",
          -5: "RP_ERR_TIMEOUT", -6: "RP_ERR_NOMEM", -7: "RP_ERR_INTERNAL", -8: "RP_ERR_SEED"}


class Request(ctypes.Structure):
    """rp_request of include/rp.h: n variates of `dist` from substream `stream`."""
    _fields_ = [("stream", ctypes.c_uint64), ("dist", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_uint64), ("p0", ctypes.c_double), ("p1", ctypes.c_double),
                ("m", ctypes.c_uint64), ("d_out", ctypes.c_void_p), ("pos", ctypes.c_uint64)]


class RPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load librp.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _build
        _build.build()
        L = ctypes.CDLL(LIB_PATH)
        u64, i32, dbl, sz, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
        pu64 = ctypes.POINTER(u64)
        sig = {
            "rp_fill_u64": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_engine_fold": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_uniform": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_uniform52": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_bounded": [i32, u64, u64, pu64, sz, u64, vp, vp],
            "rp_fill_normal": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_normal_philox_static": [u64, u64, pu64, sz, vp, vp],
            "rp_fill_exp": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_gamma": [i32, u64, u64, pu64, sz, dbl, vp, vp],
            "rp_fill_beta": [i32, u64, u64, pu64, sz, dbl, dbl, vp, vp],
            "rp_fill_derived": [i32, u64, u64, pu64, i32, ctypes.POINTER(dbl), sz, vp, vp],
            "rp_seed_state": [i32, u64, u64, pu64, ctypes.POINTER(i32)],
            "rp_jump_state": [i32, pu64, u64, u64],
            "rp_ziggurat_tables": [i32, pu64, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
            "rp_gamma_grad": [vp, dbl, vp, sz, vp, ctypes.POINTER(dbl), vp],
            "rp_fill_state": [i32, pu64, pu64, i32, sz, dbl, dbl, u64, vp, vp],
            "rp_mvn": [i32, u64, u64, pu64, i32, sz, vp, vp, vp, vp, vp],
            "rp_mvn_grads": [i32, sz, vp, vp, vp, vp, vp],
            "rp_log_cr": [vp, vp, sz, vp],
            "rp_exp_cr": [vp, vp, sz, vp],
            "rp_debug_counters": [pu64, i32],
            "rp_debug_faults": [i32, u64],
            "rp_async_status": [vp],
            "rp_fill_uniformf": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_beta_xy": [i32, u64, u64, pu64, sz, dbl, dbl, vp, vp, vp, vp],
            "rp_fill_to_host": [i32, u64, u64, pu64, i32, sz, dbl, dbl, u64, vp, vp],
            "rp_beta_grad_composed": [vp, vp, dbl, dbl, vp, sz, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp],
            "rp_fill_normalf": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_fill_expf": [i32, u64, u64, pu64, sz, vp, vp],
            "rp_substream_state": [i32, u64, u64, pu64, ctypes.POINTER(i32)],
            "rp_batch_plan_create": [ctypes.POINTER(Request), sz, i32, u64, i32, ctypes.POINTER(vp), vp],
            "rp_batch_plan_run": [vp, pu64, vp],
            "rp_batch_plan_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(dbl), pu64],
            "rp_batch_plan_destroy": [vp],
            "rp_batch_run": [ctypes.POINTER(Request), sz, i32, u64, vp],
            "rp_beta_grad": [vp, dbl, dbl, vp, sz, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i32
        L.rp_last_error.restype = ctypes.c_char_p
        L.rp_last_error.argtypes = []
        L.rp_version.restype = ctypes.c_char_p
        L.rp_version.argtypes = []
        L.rp_kernel_launches.restype = ctypes.c_uint64
        L.rp_kernel_launches.argtypes = []
        L.rp_state_serialize.restype = i32
        L.rp_state_serialize.argtypes = [i32, pu64, u64, ctypes.c_char_p, sz]
        L.rp_state_deserialize.restype = i32
        L.rp_state_deserialize.argtypes = [ctypes.c_char_p, sz, ctypes.POINTER(i32), pu64, pu64]
        L.rp_engine_name.restype = ctypes.c_char_p
        L.rp_engine_name.argtypes = [i32]
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise RPError(rc, lib().rp_last_error().decode())


def _engine(e):
    return ENGINES[e] if isinstance(e, str) else int(e)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _out(out, dtype):
    if not isinstance(out, torch.Tensor) or not out.is_cuda:
        raise TypeError("out must be a CUDA tensor")
    if out.dtype != dtype or not out.is_contiguous():
        raise TypeError(f"out must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(out.data_ptr()), out.numel()


def _pinned_pos(pos):
    """A 1-element int64/uint64 tensor in pinned host memory as a uint64*."""
    if not (pos.numel() == 1 and not pos.is_cuda and pos.is_pinned() and pos.dtype in (torch.int64, torch.uint64)):
        raise ValueError("an asynchronous position is a pinned 1-element int64/uint64 CPU tensor")
    return ctypes.cast(ctypes.c_void_p(pos.data_ptr()), ctypes.POINTER(ctypes.c_uint64))


def _fill(fn, engine, seed, stream, pos, out, dtype, extra=(), cuda_stream=None):
    """pos: an int (returns the new position after the fill completed), or a
    pinned 1-element tensor holding it (the library writes the new position
    there asynchronously; it is valid after the stream is synchronised, and
    the call returns None)."""
    p, n = _out(out, dtype)
    if isinstance(pos, torch.Tensor):
        _check(fn(_engine(engine), seed, stream, _pinned_pos(pos), n, *extra, p, _stream_handle(cuda_stream)))
        return None
    cpos = ctypes.c_uint64(pos)
    _check(fn(_engine(engine), seed, stream, ctypes.byref(cpos), n, *extra, p, _stream_handle(cuda_stream)))
    return cpos.value


def rp_async_status(cuda_stream=None):
    """Synchronises the stream and raises RPError if an asynchronous fill
    (pinned position) failed since the last check."""
    _check(lib().rp_async_status(_stream_handle(cuda_stream)))


# ---- fills: same names and argument order as the C ABI; `out` is a CUDA
# tensor of n elements; the return value is the new stream position.
def rp_fill_u64(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_u64, engine, seed, stream, pos, out, torch.uint64, cuda_stream=cuda_stream)


def rp_engine_fold(engine, seed, stream, pos, n, fold, cuda_stream=None):
    """XOR of stream words pos .. pos + n - 1 into `fold` (a 1-element uint64
    CUDA tensor); returns the new position."""
    assert fold.is_cuda and fold.dtype == torch.uint64 and fold.numel() >= 1
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_engine_fold(_engine(engine), seed, stream, ctypes.byref(cpos), n, fold.data_ptr(),
                                _stream_handle(cuda_stream)))
    return cpos.value


def rp_fill_uniform(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_uniform, engine, seed, stream, pos, out, torch.float64, cuda_stream=cuda_stream)


def rp_fill_uniform52(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_uniform52, engine, seed, stream, pos, out, torch.float64, cuda_stream=cuda_stream)


def rp_fill_bounded(engine, seed, stream, pos, m, out, cuda_stream=None):
    return _fill(lib().rp_fill_bounded, engine, seed, stream, pos, out, torch.uint64, (m,), cuda_stream)


def rp_fill_normal(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_normal, engine, seed, stream, pos, out, torch.float64, cuda_stream=cuda_stream)


STATIC_MAX_N = 1 << 22


def rp_fill_normal_philox_static(seed, stream, pos, out, cuda_stream=None):
    """Philox normal fill on the library's fixed device scratch (no
    allocation; n <= STATIC_MAX_N).  Same values as rp_fill_normal."""
    p, n = _out(out, torch.float64)
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_fill_normal_philox_static(seed, stream, ctypes.byref(cpos), n, p, _stream_handle(cuda_stream)))
    return cpos.value


def rp_fill_exp(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_exp, engine, seed, stream, pos, out, torch.float64, cuda_stream=cuda_stream)


# Float variants (suffix f): `out` a float32 CUDA tensor; the stream read as
# 32-bit words, low half of each word first.
def rp_fill_uniformf(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_uniformf, engine, seed, stream, pos, out, torch.float32, cuda_stream=cuda_stream)


def rp_fill_normalf(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_normalf, engine, seed, stream, pos, out, torch.float32, cuda_stream=cuda_stream)


def rp_fill_expf(engine, seed, stream, pos, out, cuda_stream=None):
    return _fill(lib().rp_fill_expf, engine, seed, stream, pos, out, torch.float32, cuda_stream=cuda_stream)


def rp_fill_gamma(engine, seed, stream, pos, alpha, out, cuda_stream=None):
    return _fill(lib().rp_fill_gamma, engine, seed, stream, pos, out, torch.float64, (float(alpha),), cuda_stream)


def rp_fill_beta(engine, seed, stream, pos, a, b, out, cuda_stream=None):
    return _fill(lib().rp_fill_beta, engine, seed, stream, pos, out, torch.float64, (float(a), float(b)),
                 cuda_stream)


# Derived distributions (Table "continuous"): name -> (rp_derived code,
# parameter names); see rp_fill_derived in include/rp.h for the formulas.
DERIVED = {"unif": (1, ("a", "b")), "normal_ms": (2, ("mu", "sigma")), "lognormal": (3, ("mu", "sigma")),
           "exp_scale": (4, ("beta",)), "gamma_scale": (5, ("alpha", "theta")), "chi2": (6, ("nu",)),
           "gumbel": (7, ("mu", "beta")), "pareto": (8, ("x_m", "alpha")), "weibull": (9, ("k", "lambda")),
           "gpd": (10, ("mu", "sigma", "xi")), "f": (11, ("nu1", "nu2")), "skew_normal": (12, ("mu", "sigma", "alpha")),
           "t": (13, ("nu",))}


def rp_fill_derived(engine, seed, stream, pos, name, params, out, cuda_stream=None):
    """Fill `out` (float64 CUDA tensor) with a derived distribution `name`
    (a key of DERIVED) and its parameters; returns the new stream position."""
    kind, names = DERIVED[name]
    if len(params) != len(names):
        raise ValueError(f"{name} takes {names}")
    p, n = _out(out, torch.float64)
    q = (ctypes.c_double * 4)(*([float(x) for x in params] + [0.0] * (4 - len(params))))
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_fill_derived(_engine(engine), seed, stream, ctypes.byref(cpos), kind, q, n, p,
                                 _stream_handle(cuda_stream)))
    return cpos.value


def _ptr_or_null(t, n):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError("size mismatch")
    return ctypes.c_void_p(t.data_ptr())


def rp_gamma_grad(z, alpha, g=None, dzda=None, cuda_stream=None):
    """Pathwise gradient of Gamma(alpha) variates z: fills dzda (optional) with
    dz/dalpha and returns sum(g * dz/dalpha) (None without g)."""
    n = z.numel()
    out = ctypes.c_double()
    _check(lib().rp_gamma_grad(_ptr_or_null(z, n), float(alpha), _ptr_or_null(g, n), n, _ptr_or_null(dzda, n),
                               ctypes.byref(out), _stream_handle(cuda_stream)))
    return out.value if g is not None else None


def rp_beta_grad(z, a, b, g=None, dzda=None, dzdb=None, cuda_stream=None):
    """Pathwise gradient of Beta(a, b) variates z: dz/da, dz/db per sample
    (optional) and the sums with g (None without g)."""
    n = z.numel()
    ga, gb = ctypes.c_double(), ctypes.c_double()
    _check(lib().rp_beta_grad(_ptr_or_null(z, n), float(a), float(b), _ptr_or_null(g, n), n, _ptr_or_null(dzda, n),
                              _ptr_or_null(dzdb, n), ctypes.byref(ga), ctypes.byref(gb), _stream_handle(cuda_stream)))
    return (ga.value, gb.value) if g is not None else None


def rp_fill_to_host(engine, seed, stream, pos, dist, out, p0=0.0, p1=0.0, m=0, cuda_stream=None):
    """rp_fill_state's distribution `dist` (a DIST name or code), seeded, into
    `out`, a CPU tensor of 8-byte elements (pinned: asynchronous, complete
    after torch.cuda.synchronize()).  pos: an int (returns the new position)
    or a pinned 1-element tensor (written asynchronously; returns None)."""
    if out.is_cuda or out.element_size() != 8 or not out.is_contiguous():
        raise TypeError("out must be a contiguous CPU tensor of 8-byte elements")
    d = DISTS[dist] if isinstance(dist, str) else int(dist)
    args = (_engine(engine), seed, stream)
    tail = (d, out.numel(), float(p0), float(p1), int(m), ctypes.c_void_p(out.data_ptr()), _stream_handle(cuda_stream))
    if isinstance(pos, torch.Tensor):
        _check(lib().rp_fill_to_host(*args, _pinned_pos(pos), *tail))
        return None
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_fill_to_host(*args, ctypes.byref(cpos), *tail))
    return cpos.value


def rp_fill_beta_xy(engine, seed, stream, pos, a, b, z, x, y, cuda_stream=None):
    """rp_fill_beta that also keeps each output's gamma pair in x and y
    (float64 CUDA tensors of the same length); returns the new position."""
    p, n = _out(z, torch.float64)
    px, nx = _out(x, torch.float64)
    py, ny = _out(y, torch.float64)
    if nx != n or ny != n:
        raise ValueError("z, x and y must have the same length")
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_fill_beta_xy(_engine(engine), seed, stream, ctypes.byref(cpos), n, float(a), float(b), p, px, py,
                                 _stream_handle(cuda_stream)))
    return cpos.value


def rp_beta_grad_composed(x, y, a, b, g=None, dzda=None, dzdb=None, cuda_stream=None):
    """Beta gradient through the gamma pairs (x, y): dz/da, dz/db per sample
    (optional) and the sums with g (None without g)."""
    n = x.numel()
    ga, gb = ctypes.c_double(), ctypes.c_double()
    _check(lib().rp_beta_grad_composed(_ptr_or_null(x, n), _ptr_or_null(y, n), float(a), float(b), _ptr_or_null(g, n), n,
                                       _ptr_or_null(dzda, n), _ptr_or_null(dzdb, n), ctypes.byref(ga), ctypes.byref(gb),
                                       _stream_handle(cuda_stream)))
    return (ga.value, gb.value) if g is not None else None


class Gamma(torch.autograd.Function):
    """z ~ Gamma(alpha, 1) (n draws from the given stream), differentiable in
    alpha by the pathwise (implicit CDF) gradient computed in librp.
    Gamma.apply(alpha, n, engine, seed, stream, pos) -> z; the new stream
    position is left in Gamma.last_pos."""
    last_pos = None

    @staticmethod
    def forward(ctx, alpha, n, engine, seed, stream, pos):
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        Gamma.last_pos = rp_fill_gamma(engine, seed, stream, pos, float(alpha), z)
        ctx.save_for_backward(z)
        ctx.alpha = float(alpha)
        return z

    @staticmethod
    def backward(ctx, grad_z):
        (z,) = ctx.saved_tensors
        ga = rp_gamma_grad(z, ctx.alpha, grad_z.to(torch.float64).contiguous())
        return torch.tensor(ga, dtype=torch.float64), None, None, None, None, None


class Beta(torch.autograd.Function):
    """z ~ Beta(a, b), differentiable in a and b (pathwise gradient).
    Beta.apply(a, b, n, engine, seed, stream, pos) -> z; new position in
    Beta.last_pos."""
    last_pos = None

    @staticmethod
    def forward(ctx, a, b, n, engine, seed, stream, pos):
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        Beta.last_pos = rp_fill_beta(engine, seed, stream, pos, float(a), float(b), z)
        ctx.save_for_backward(z)
        ctx.ab = (float(a), float(b))
        return z

    @staticmethod
    def backward(ctx, grad_z):
        (z,) = ctx.saved_tensors
        ga, gb = rp_beta_grad(z, ctx.ab[0], ctx.ab[1], grad_z.to(torch.float64).contiguous())
        return torch.tensor(ga, dtype=torch.float64), torch.tensor(gb, dtype=torch.float64), None, None, None, None, None


def _dist(d):
    return DISTS[d] if isinstance(d, str) else int(d)


def rp_fill_state(engine, words, pos, dist, out, p0=0.0, p1=0.0, m=0, cuda_stream=None):
    """Fill `out` from a stream given by its state words (before word 0),
    starting at word `pos`; returns the next unused word."""
    w = (ctypes.c_uint64 * 4)(*[int(x) for x in list(words) + [0] * (4 - len(words))])
    d = _dist(dist)
    p, n = _out(out, torch.uint64 if d in (0, 2) else torch.float64)
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_fill_state(_engine(engine), w, ctypes.byref(cpos), d, n, float(p0), float(p1), int(m), p,
                               _stream_handle(cuda_stream)))
    return cpos.value


STATE_BYTES = 64


def rp_state_serialize(engine, words, pos):
    """A stream's state (engine, state words before word 0, position) as the
    library's opaque checkpoint bytes."""
    w = (ctypes.c_uint64 * 4)(*[int(x) for x in list(words) + [0] * (4 - len(words))])
    buf = ctypes.create_string_buffer(STATE_BYTES)
    _check(lib().rp_state_serialize(_engine(engine), w, pos, buf, STATE_BYTES))
    return buf.raw


def rp_state_deserialize(data):
    """(engine id, four state words, position) from checkpoint bytes."""
    e = ctypes.c_int()
    w = (ctypes.c_uint64 * 4)()
    p = ctypes.c_uint64()
    _check(lib().rp_state_deserialize(bytes(data), len(data), ctypes.byref(e), w, ctypes.byref(p)))
    return e.value, [w[i] for i in range(4)], p.value


def rp_engine_name(engine):
    r = lib().rp_engine_name(int(engine))
    return None if r is None else r.decode()


def rp_substream_state(engine, base_seed, s):
    """State words of substream s of base_seed (Sec. 2.3 recipe)."""
    w = (ctypes.c_uint64 * 4)()
    nw = ctypes.c_int()
    _check(lib().rp_substream_state(_engine(engine), base_seed, s, w, ctypes.byref(nw)))
    return [w[i] for i in range(nw.value)]


def make_requests(specs):
    """Request array from dicts with keys stream, dist, out (CUDA tensor) and
    optional p0, p1, m, pos."""
    arr = (Request * len(specs))()
    for i, sp in enumerate(specs):
        out = sp["out"]
        if not isinstance(out, torch.Tensor) or not out.is_cuda or out.element_size() != 8 or not out.is_contiguous():
            raise TypeError("request outputs must be contiguous 8-byte CUDA tensors")
        arr[i] = Request(int(sp["stream"]), _dist(sp["dist"]), 0, out.numel(), float(sp.get("p0", 0.0)),
                         float(sp.get("p1", 0.0)), int(sp.get("m", 0)), out.data_ptr() if out.numel() else None,
                         int(sp.get("pos", 0)))
    return arr


class BatchPlan:
    """A batch plan (rp_batch_plan_*): one CUDA-graph launch serves every
    request; run() returns each request's next unused word."""

    def __init__(self, reqs, engine, base_seed, autotune=False, cuda_stream=None):
        self._reqs = reqs
        self.n = len(reqs)
        h = ctypes.c_void_p()
        _check(lib().rp_batch_plan_create(reqs, self.n, _engine(engine), base_seed, int(bool(autotune)),
                                          ctypes.byref(h), _stream_handle(cuda_stream)))
        self._h = h

    def run(self, cuda_stream=None):
        np_ = (ctypes.c_uint64 * max(self.n, 1))()
        _check(lib().rp_batch_plan_run(self._h, np_, _stream_handle(cuda_stream)))
        return [np_[i] for i in range(self.n)]

    def info(self):
        sch, ms, it = ctypes.c_int(), ctypes.c_double(), ctypes.c_uint64()
        _check(lib().rp_batch_plan_info(self._h, ctypes.byref(sch), ctypes.byref(ms), ctypes.byref(it)))
        return {"schedule": sch.value, "tuned_ms": ms.value, "items": it.value}

    def close(self):
        if self._h:
            lib().rp_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rp_batch_run(reqs, engine, base_seed, cuda_stream=None):
    """One-shot batch: fills every request; returns the next unused words."""
    _check(lib().rp_batch_run(reqs, len(reqs), _engine(engine), base_seed, _stream_handle(cuda_stream)))
    return [reqs[i].pos for i in range(len(reqs))]


def _f64(t, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else None


def rp_mvn(engine, seed, stream, pos, mu, L, Z, X, cuda_stream=None):
    """X = mu + L z per sample, z from the normal stream (Z saved, n x d);
    returns the next unused word."""
    n, d = X.shape
    cpos = ctypes.c_uint64(pos)
    _check(lib().rp_mvn(_engine(engine), seed, stream, ctypes.byref(cpos), d, n, _f64(mu, (d,), "mu"),
                        _f64(L, (d, d), "L"), _f64(Z, (n, d), "Z"), _f64(X, (n, d), "X"),
                        _stream_handle(cuda_stream)))
    return cpos.value


def rp_mvn_grads(G, Z, gmu, gL, cuda_stream=None):
    """dL/dmu = sum_j G_j, dL/dL = tril(G^T Z)."""
    n, d = Z.shape
    _check(lib().rp_mvn_grads(d, n, _f64(G, (n, d), "G"), _f64(Z, (n, d), "Z"), _f64(gmu, (d,), "gmu"),
                              _f64(gL, (d, d), "gL"), _stream_handle(cuda_stream)))


class MVN(torch.autograd.Function):
    """x = mu + L z (n samples), differentiable in mu and L (lower triangle).
    MVN.apply(mu, L, n, engine, seed, stream, pos) -> X (n x d); the next
    stream word is left in MVN.last_pos."""
    last_pos = None

    @staticmethod
    def forward(ctx, mu, L, n, engine, seed, stream, pos):
        d = mu.shape[0]
        Z = torch.empty((n, d), dtype=torch.float64, device="cuda")
        X = torch.empty((n, d), dtype=torch.float64, device="cuda")
        MVN.last_pos = rp_mvn(engine, seed, stream, pos, mu.detach().contiguous(), L.detach().contiguous(), Z, X)
        ctx.save_for_backward(Z)
        return X

    @staticmethod
    def backward(ctx, G):
        (Z,) = ctx.saved_tensors
        n, d = Z.shape
        gmu = torch.empty(d, dtype=torch.float64, device="cuda")
        gL = torch.empty((d, d), dtype=torch.float64, device="cuda")
        rp_mvn_grads(G.to(torch.float64).contiguous(), Z, gmu, gL)
        return gmu, gL, None, None, None, None, None


DEBUG_COUNTERS = ("wedge_fp64", "wedge_cr", "tail_fp64", "tail_cr", "mt_fp64", "mt_cr")


def rp_debug_counters(reset=False):
    """Fallback counts of the exact accept decisions since the last reset, as
    a dict over DEBUG_COUNTERS."""
    c = (ctypes.c_uint64 * 6)()
    _check(lib().rp_debug_counters(c, 1 if reset else 0))
    return dict(zip(DEBUG_COUNTERS, (int(x) for x in c)))


FAULTS = {"clear": 0, "spin_max": 1, "stall_tile": 2, "tail_cap": 3, "tile_cap": 4}


def rp_debug_faults(kind, value=0):
    """Set a test hook of the device error paths (see include/rp.h); kind is
    a key of FAULTS or its number."""
    _check(lib().rp_debug_faults(FAULTS.get(kind, kind), int(value)))


def rp_exp_cr(x, y=None, cuda_stream=None):
    """Correctly rounded exp of a float64 CUDA tensor (element-wise)."""
    if y is None:
        y = torch.empty_like(x)
    n = x.numel()
    _check(lib().rp_exp_cr(_f64(x, x.shape, "x"), _f64(y, x.shape, "y"), n, _stream_handle(cuda_stream)))
    return y


def rp_log_cr(x, y=None, cuda_stream=None):
    """Correctly rounded log of a float64 CUDA tensor (element-wise)."""
    if y is None:
        y = torch.empty_like(x)
    n = x.numel()
    _check(lib().rp_log_cr(_f64(x, x.shape, "x"), _f64(y, x.shape, "y"), n, _stream_handle(cuda_stream)))
    return y


def rp_seed_state(engine, seed, stream=NO_STREAM):
    w = (ctypes.c_uint64 * 4)()
    nw = ctypes.c_int()
    _check(lib().rp_seed_state(_engine(engine), seed, stream, w, ctypes.byref(nw)))
    return [int(x) for x in w[: nw.value]]


def rp_jump_state(engine, words, delta):
    w = (ctypes.c_uint64 * 4)(*(list(words) + [0] * (4 - len(words))))
    _check(lib().rp_jump_state(_engine(engine), w, (delta >> 64) & (2 ** 64 - 1), delta & (2 ** 64 - 1)))
    return [int(x) for x in w[: len(words)]]


def rp_ziggurat_tables(which):
    k = (ctypes.c_uint64 * 256)()
    w = (ctypes.c_double * 256)()
    f = (ctypes.c_double * 256)()
    R = ctypes.c_double()
    _check(lib().rp_ziggurat_tables(which, k, w, f, ctypes.byref(R)))
    return list(k), list(w), list(f), R.value


def rp_last_error():
    return lib().rp_last_error().decode()


def rp_version():
    return lib().rp_version().decode()


def rp_kernel_launches():
    return int(lib().rp_kernel_launches())


# ---- convenience: allocate and fill
_DIST_DTYPE = {"u64": torch.uint64, "uniform": torch.float64, "uniform52": torch.float64, "bounded": torch.uint64,
               "normal": torch.float64, "exp": torch.float64, "gamma": torch.float64, "beta": torch.float64}


def fill(dist, n, engine="xoshiro256pp", seed=0, stream=NO_STREAM, pos=0, params=(), out=None, cuda_stream=None):
    """Allocate (unless `out` is given) and fill n variates; returns (out, new_pos)."""
    if out is None:
        out = torch.empty(n, dtype=_DIST_DTYPE.get(dist, torch.float64), device="cuda")
    f = {"u64": rp_fill_u64, "uniform": rp_fill_uniform, "uniform52": rp_fill_uniform52, "normal": rp_fill_normal,
         "exp": rp_fill_exp}
    if dist in f:
        newpos = f[dist](engine, seed, stream, pos, out, cuda_stream)
    elif dist == "bounded":
        newpos = rp_fill_bounded(engine, seed, stream, pos, params[0], out, cuda_stream)
    elif dist == "gamma":
        newpos = rp_fill_gamma(engine, seed, stream, pos, params[0], out, cuda_stream)
    elif dist == "beta":
        newpos = rp_fill_beta(engine, seed, stream, pos, params[0], params[1], out, cuda_stream)
    elif dist in DERIVED:
        newpos = rp_fill_derived(engine, seed, stream, pos, dist, params, out, cuda_stream)
    else:
        raise ValueError(dist)
    return out, newpos
