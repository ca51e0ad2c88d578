"""Philox normal fill on fixed static scratch (rp_fill_normal_philox_static)
against the allocating entry point rp_fill_normal, both called through the
C ABI: two calls in a row, the second continuing from the first's position,
each bit-identical to rp_fill_normal from the same position (both run the
same kernels, tail values included, so any misplaced entry of the fixed
array shows).  Sizes above RP_STATIC_MAX_N are refused before any device
work.  Collected last so that it also runs after every other test in one
process."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2605_05099_gb300 as rp

pytestmark = pytest.mark.gpu

MAX_N = 1 << 22


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _static(seed, stream, pos, out):
    """Direct C-ABI call; returns (status, new position)."""
    cpos = ctypes.c_uint64(pos)
    rc = rp.lib().rp_fill_normal_philox_static(seed, stream, ctypes.byref(cpos), out.numel(),
                                              ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, cpos.value


def _reference(seed, stream, pos, n):
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    cpos = ctypes.c_uint64(pos)
    rc = rp.lib().rp_fill_normal(3, seed, stream, ctypes.byref(cpos), n, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rp.lib().rp_last_error()
    return out.cpu().numpy(), cpos.value


def _assert_identical(got, ref):
    bad = np.nonzero(got.view(np.int64) != ref.view(np.int64))[0]
    assert len(bad) == 0, (len(bad), bad[:8])


@pytest.mark.parametrize("seed,stream,pos0,n1,n2", [
    (2024, rp.NO_STREAM, 0, 100003, MAX_N),
    (7, 5, 12345, 1, 8193),
])
def test_two_calls_in_a_row_match_allocating_fill(seed, stream, pos0, n1, n2):
    a = torch.full((n1,), float("nan"), dtype=torch.float64, device="cuda")
    b = torch.full((n2,), float("nan"), dtype=torch.float64, device="cuda")
    rc, p1 = _static(seed, stream, pos0, a)
    assert rc == 0, rp.lib().rp_last_error()
    rc, p2 = _static(seed, stream, p1, b)
    assert rc == 0, rp.lib().rp_last_error()
    torch.cuda.synchronize()
    ra, q1 = _reference(seed, stream, pos0, n1)
    rb, q2 = _reference(seed, stream, q1, n2)
    assert (p1, p2) == (q1, q2)
    ga, gb = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(np.isfinite(ga)) and np.all(np.isfinite(gb))
    _assert_identical(ga, ra)
    _assert_identical(gb, rb)


def test_size_above_limit_is_refused():
    out = torch.full((MAX_N + 1,), float("nan"), dtype=torch.float64, device="cuda")
    rc, p = _static(1, rp.NO_STREAM, 77, out)
    assert rc == -2
    assert "RP_STATIC_MAX_N" in rp.lib().rp_last_error().decode()
    assert p == 77
    torch.cuda.synchronize()
    assert torch.isnan(out).all().item()


def test_binding_and_null_position():
    out = torch.empty(1000, dtype=torch.float64, device="cuda")
    p = rp.rp_fill_normal_philox_static(3, rp.NO_STREAM, 0, out)
    ref, q = _reference(3, rp.NO_STREAM, 0, 1000)
    assert p == q
    _assert_identical(out.cpu().numpy(), ref)
    assert rp.lib().rp_fill_normal_philox_static(3, rp.NO_STREAM, None, 10, ctypes.c_void_p(out.data_ptr()),
                                                None) == -1
