"""C-ABI checks that need no GPU: the library loads, exports every symbol
that include/rp.h declares, and its host-side logic (seeding, jumps, tables,
argument validation) agrees with the oracle.  No compute call reaches CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rp():
    import paper_2605_05099_gb300 as rp
    rp.lib()
    return rp


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "rp.h")).read()
    return sorted(set(re.findall(r"\b(rp_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(rp):
    syms = _declared_symbols()
    assert len(syms) >= 12
    L = rp.lib()
    for s in syms:
        assert hasattr(L, s), s


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10", "philox4x64_10", "xoshiro256ss"])
def test_seed_state_matches_oracle(rp, orc, engine):
    rng = np.random.default_rng(5)
    for seed in [0, 1, 7, 99, 2024, 12345, 2 ** 40 + 3, 2 ** 64 - 1] + [int(x) for x in rng.integers(0, 2 ** 62, 20)]:
        for stream in [None, 0, 1, 2 ** 33]:
            g = orc.gen(engine, seed, stream)
            w = rp.rp_seed_state(engine, seed, rp.NO_STREAM if stream is None else stream)
            assert w == orc.state_words(g)[: len(w)], (engine, seed, stream)


def test_jump_state_matches_oracle(rp, orc):
    rng = np.random.default_rng(6)
    s0 = rp.rp_seed_state("xoshiro256pp", 99)
    for n in [1, 2, 1000, 2 ** 64 - 1, 2 ** 128 - 5] + [int(x) for x in rng.integers(0, 2 ** 62, 5)]:
        assert rp.rp_jump_state("xoshiro256pp", s0, n) == orc.xoshiro_jump(s0, n, "matrix" if n < 2 ** 70 else "poly")
    p0 = rp.rp_seed_state("pcg64dxsm", 5)
    for n in [1, 3, 2 ** 64 + 17, int(rng.integers(0, 2 ** 62))]:
        assert rp.rp_jump_state("pcg64dxsm", p0, n) == orc.pcg_advance(p0, n)
    ph = rp.rp_seed_state("philox4x32_10", 3)
    j = rp.rp_jump_state("philox4x32_10", ph, 2 ** 65 + 10)
    c0, c1 = ph[0] | ph[1] << 64, j[0] | j[1] << 64
    assert c1 - c0 == 2 ** 64 + 5 and j[2] == ph[2]
    # xoshiro256** jumps with xoshiro256++'s tables (one transition)
    x = rp.rp_seed_state("xoshiro256ss", 99)
    assert x == s0 and rp.rp_jump_state("xoshiro256ss", x, 2 ** 100 + 3) == orc.xoshiro_jump(s0, 2 ** 100 + 3, "poly")
    q = rp.rp_seed_state("philox4x64_10", 3)
    j = rp.rp_jump_state("philox4x64_10", q, 2 ** 66 + 12)   # four words per block
    assert (j[0] | j[1] << 64) - (q[0] | q[1] << 64) == 2 ** 64 + 3 and j[2:] == q[2:]
    with pytest.raises(rp.RPError):
        rp.rp_jump_state("philox4x64_10", q, 6)


def test_ziggurat_tables_match_oracle(rp, orc):
    for which in (0, 1):
        k, w, f, R = rp.rp_ziggurat_tables(which)
        ok, ow, of, oR = orc.zig_table(which)
        assert [int(x) for x in ok] == k
        assert list(ow) == w and list(of) == f and oR == R


def test_argument_errors(rp):
    L = rp.lib()
    pos = ctypes.c_uint64(0)
    dummy = ctypes.c_void_p(0x1000)
    # null pos, null out with n > 0, bad engine, misaligned out, bad params
    assert L.rp_fill_u64(1, 1, rp.NO_STREAM, None, 10, dummy, None) == -1
    assert L.rp_fill_u64(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, None, None) == -1
    assert L.rp_fill_normal(9, 1, rp.NO_STREAM, ctypes.byref(pos), 10, dummy, None) == -3
    assert "engine" in rp.rp_last_error()
    assert L.rp_fill_exp(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, ctypes.c_void_p(0x1004), None) == -2
    assert L.rp_fill_gamma(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, 0.0, dummy, None) == -2
    assert L.rp_fill_gamma(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, float("nan"), dummy, None) == -2
    assert L.rp_fill_beta(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, 1.0, -2.0, dummy, None) == -2
    assert L.rp_seed_state(1, 1, 0, None, None) == -1
    assert L.rp_jump_state(3, (ctypes.c_uint64 * 4)(), 0, 3) == -2  # odd Philox state jump
    # n = 0 is a no-op that leaves pos alone (no device work)
    pos = ctypes.c_uint64(77)
    for fn in (L.rp_fill_u64, L.rp_fill_uniform, L.rp_fill_normal, L.rp_fill_exp):
        assert fn(1, 1, rp.NO_STREAM, ctypes.byref(pos), 0, None, None) == 0
    assert pos.value == 77
    assert rp.rp_version().startswith("rp ")


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10", "philox4x64_10", "xoshiro256ss"])
def test_substream_state_matches_oracle(rp, orc, engine):
    """Substream s of a base seed (Sec. 2.3 recipe): library host code vs the
    oracle's independent construction (xoshiro: jump polynomial by s 2^128)."""
    for s in [0, 1, 2, 5, 4095, 2**40 + 7]:
        w = rp.rp_substream_state(engine, 99, s)
        ow = orc.state_words(orc.substream(engine, 99, s))
        assert w == ow[:len(w)], (engine, s)


def test_batch_argument_errors_without_device(rp):
    L = rp.lib()
    import ctypes
    assert L.rp_batch_plan_create(None, 0, 1, 99, 0, None, None) == -1
    assert L.rp_batch_plan_run(None, None, None) == -1
    assert L.rp_batch_plan_info(None, None, None, None) == -1
    assert L.rp_fill_state(1, None, None, 3, 5, 0.0, 0.0, 0, None, None) == -1
    w = (ctypes.c_uint64 * 4)(1, 2, 3, 4)
    p = ctypes.c_uint64(0)
    assert L.rp_fill_state(7, w, ctypes.byref(p), 3, 5, 0.0, 0.0, 0, ctypes.c_void_p(0x1000), None) == -3
    assert L.rp_substream_state(9, 99, 1, w, ctypes.byref(ctypes.c_int())) == -3


def test_derived_argument_errors_without_device(rp):
    """rp_fill_derived refuses bad parameters and unknown kinds before any
    device work; its codes match the header's enum and the binding's table."""
    import ctypes
    import re
    L = rp.lib()
    p = ctypes.c_uint64(0)
    q = (ctypes.c_double * 4)(1.0, 0.0, 0.0, 0.0)
    assert L.rp_fill_derived(1, 1, 0, ctypes.byref(p), 1, q, 5, None, None) == -2      # unif with a > b
    assert L.rp_fill_derived(1, 1, 0, ctypes.byref(p), 2, q, 5, None, None) == -2      # sigma = 0
    assert L.rp_fill_derived(1, 1, 0, ctypes.byref(p), 99, q, 5, None, None) == -2     # unknown kind
    assert L.rp_fill_derived(1, 1, 0, ctypes.byref(p), 1, None, 5, None, None) == -1   # no parameters
    hdr = open(os.path.join(ROOT, "include", "rp.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} rp_derived;", hdr).group(1)
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"RP_(\w+) = (\d+)", body)}
    import oracle
    for name, (kind, _) in rp.DERIVED.items():
        assert codes[name.upper()] == kind and oracle.DERIVED[name][0] == kind, name


@pytest.mark.parametrize("engine", ["xoshiro256pp", "pcg64dxsm", "philox4x32_10", "philox4x64_10", "xoshiro256ss"])
def test_state_checkpoint_round_trip(rp, orc, engine):
    """A serialised state (Sec. 4.4 checkpointing) restores exactly, and any
    single corrupted byte, a short buffer or an unknown engine is refused."""
    words = rp.rp_seed_state(engine, 2024, 3)
    for pos in (0, 1, 2 ** 40 + 7, 2 ** 64 - 1):
        buf = rp.rp_state_serialize(engine, words, pos)
        assert len(buf) == rp.STATE_BYTES
        e, w, p = rp.rp_state_deserialize(buf)
        assert e == rp.ENGINES[engine] and w[:len(words)] == words and p == pos
        for i in range(rp.STATE_BYTES):
            bad = bytearray(buf)
            bad[i] ^= 0x10
            with pytest.raises(rp.RPError):
                rp.rp_state_deserialize(bytes(bad))
    with pytest.raises(rp.RPError):
        rp.rp_state_deserialize(buf[:-1])
    with pytest.raises(rp.RPError):
        rp.rp_state_serialize(9, words, 0)
    assert rp.rp_engine_name(rp.ENGINES[engine]) == engine and rp.rp_engine_name(0) is None


def test_dist_codes_match_the_header(rp):
    """The binding's distribution codes are rp.h's rp_dist values."""
    import re
    hdr = open(os.path.join(ROOT, "include", "rp.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} rp_dist;", hdr).group(1)
    codes = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"RP_DIST_(\w+) = (\d+)", body)}
    assert codes == rp.DISTS


def test_engine_codes_match_the_header(rp, orc):
    """rp.h's rp_engine values are the binding's and the oracle's engine ids."""
    import re
    hdr = open(os.path.join(ROOT, "include", "rp.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} rp_engine;", hdr).group(1)
    codes = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"RP_(\w+) = (\d+)", body)}
    assert codes == rp.ENGINES == orc.ENGINES
    for name, e in codes.items():
        assert rp.rp_engine_name(e) == name


def test_binding_refuses_bad_outputs_before_the_library(rp):
    """The Python binding checks the output tensor (device, dtype, layout) and
    the derived law's parameter count before any call into librp."""
    import torch
    cpu = torch.empty(8, dtype=torch.float64)
    with pytest.raises(TypeError):
        rp.rp_fill_normal("xoshiro256pp", 1, rp.NO_STREAM, 0, cpu)
    with pytest.raises(ValueError):
        rp.rp_fill_derived("xoshiro256pp", 1, rp.NO_STREAM, 0, "gumbel", (1.0,), cpu)
    with pytest.raises(KeyError):
        rp.rp_fill_derived("xoshiro256pp", 1, rp.NO_STREAM, 0, "no_such_law", (1.0,), cpu)
    with pytest.raises(KeyError):
        rp.rp_seed_state("no_such_engine", 1)


def test_last_error_is_per_host_thread(rp):
    """rp_last_error returns the calling thread's last failure (the header's
    convention, after the per-generator error string of Sec. 2.1): two
    threads that fail differently each read back their own message."""
    import ctypes
    import threading
    L = rp.lib()
    got = {}
    barrier = threading.Barrier(2)

    def fail_engine():
        pos = ctypes.c_uint64(0)
        assert L.rp_fill_normal(9, 1, rp.NO_STREAM, ctypes.byref(pos), 10, ctypes.c_void_p(0x1000), None) == -3
        barrier.wait()
        got["engine"] = rp.rp_last_error()

    def fail_param():
        pos = ctypes.c_uint64(0)
        assert L.rp_fill_gamma(1, 1, rp.NO_STREAM, ctypes.byref(pos), 10, -1.0, ctypes.c_void_p(0x1000), None) == -2
        barrier.wait()
        got["param"] = rp.rp_last_error()

    ts = [threading.Thread(target=fail_engine), threading.Thread(target=fail_param)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert got["engine"] == "unknown engine id 9"
    assert got["param"] == "gamma shape must be positive and finite"


def _fnv1a64(data):
    """FNV-1a, 64-bit (offset basis 0xcbf29ce484222325, prime 0x100000001b3)."""
    h = 0xCBF29CE484222325
    for b in data:
        h = ((h ^ b) * 0x100000001B3) & (2 ** 64 - 1)
    return h


def _state_buf(magic=b"RPST", version=1, engine=1, words=(1, 2, 3, 4), pos=5, reserved=0):
    import struct
    head = magic + struct.pack("<HH4QQQ", version, engine, *words, pos, reserved)
    return head + struct.pack("<Q", _fnv1a64(head))


def test_checkpoint_layout_is_the_documented_one(rp):
    """The 64-byte layout of rp.h, written here byte by byte with an
    independent FNV-1a: a library-written buffer equals it, and buffers with
    a valid checksum are still refused for a wrong magic or version, an
    unknown engine, nonzero reserved bytes or an all-zero xoshiro state."""
    words = rp.rp_seed_state("xoshiro256ss", 2024, 3)
    assert rp.rp_state_serialize("xoshiro256ss", words, 77) == _state_buf(engine=5, words=words, pos=77)
    assert rp.rp_state_deserialize(_state_buf()) == (1, [1, 2, 3, 4], 5)
    for bad in (_state_buf(magic=b"RPSX"), _state_buf(version=2), _state_buf(engine=6), _state_buf(engine=0),
                _state_buf(reserved=1), _state_buf(engine=1, words=(0, 0, 0, 0)),
                _state_buf(engine=5, words=(0, 0, 0, 0))):
        with pytest.raises(rp.RPError):
            rp.rp_state_deserialize(bad)
    # PCG and Philox states may be all zero
    assert rp.rp_state_deserialize(_state_buf(engine=3, words=(0, 0, 0, 0)))[0] == 3


def test_gradient_and_mvn_argument_errors_without_device(rp):
    """Gradients and the MVN entry points check their arguments before any
    device work: bad shapes and missing pointers are refused, and n = 0
    returns zero sums without touching the device."""
    import ctypes
    L = rp.lib()
    dummy = ctypes.c_void_p(0x1000)
    h = ctypes.c_double(7.0)
    h2 = ctypes.c_double(7.0)
    assert L.rp_gamma_grad(dummy, ctypes.c_double(0.0), dummy, 4, None, ctypes.byref(h), None) == -2
    assert L.rp_gamma_grad(dummy, ctypes.c_double(float("inf")), dummy, 4, None, ctypes.byref(h), None) == -2
    assert L.rp_gamma_grad(None, ctypes.c_double(2.0), dummy, 4, None, ctypes.byref(h), None) == -1
    assert L.rp_gamma_grad(dummy, ctypes.c_double(2.0), dummy, 4, None, None, None) == -1
    assert L.rp_gamma_grad(dummy, ctypes.c_double(2.0), None, 4, None, None, None) == -1
    assert L.rp_gamma_grad(None, ctypes.c_double(2.0), None, 0, None, ctypes.byref(h), None) == 0 and h.value == 0.0
    assert L.rp_beta_grad(dummy, ctypes.c_double(-1.0), ctypes.c_double(2.0), dummy, 4, None, None,
                          ctypes.byref(h), ctypes.byref(h2), None) == -2
    assert L.rp_beta_grad(dummy, ctypes.c_double(1.0), ctypes.c_double(2.0), dummy, 4, None, None,
                          ctypes.byref(h), None, None) == -1
    h.value = h2.value = 7.0
    assert L.rp_beta_grad(None, ctypes.c_double(1.0), ctypes.c_double(2.0), None, 0, None, None,
                          ctypes.byref(h), ctypes.byref(h2), None) == 0 and h.value == 0.0 and h2.value == 0.0
    pos = ctypes.c_uint64(11)
    assert L.rp_mvn(1, 3, rp.NO_STREAM, ctypes.byref(pos), 0, 8, dummy, dummy, dummy, dummy, None) == -2
    assert L.rp_mvn(1, 3, rp.NO_STREAM, None, 4, 8, dummy, dummy, dummy, dummy, None) == -1
    assert L.rp_mvn(1, 3, rp.NO_STREAM, ctypes.byref(pos), 4, 8, None, dummy, dummy, dummy, None) == -1
    assert L.rp_mvn(1, 3, rp.NO_STREAM, ctypes.byref(pos), 4, 0, None, None, None, None, None) == 0 and pos.value == 11
    assert L.rp_mvn_grads(0, 8, dummy, dummy, dummy, dummy, None) == -2
    assert L.rp_mvn_grads(4, 8, None, dummy, dummy, dummy, None) == -1
