"""Device error paths, made to fail on purpose through host-set test hooks
(rp_debug_faults) and never by faulting or hanging the GPU: a look-back
wait that runs out (one tile never publishes its count, the others give up
after a few thousand spins), a tail queue too small for the fill, and a
fill that needs more continuation launches than allowed.  Each reports its
error code, and a fill right after it on the same stream is bit-exact
again (Sec. 2.1: errors are returned, never aborted on)."""
import numpy as np
import pytest
import torch

import paper_2605_05099_gb300 as rp
from gpu_util import assert_parity, gpu_fill

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clear_faults():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rp.rp_debug_faults("clear")
    yield
    rp.rp_debug_faults("clear")


def _fails(code, dist, engine, n):
    with pytest.raises(rp.RPError) as ei:
        gpu_fill(dist, engine, 2024, None, 0, n)
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


@pytest.mark.parametrize("engine,dist", [("xoshiro256pp", "normal"), ("philox4x32_10", "exp")])
def test_lookback_wait_runs_out(engine, dist):
    rp.rp_debug_faults("spin_max", 2000)
    rp.rp_debug_faults("stall_tile", 5)          # tile 4 never publishes
    _fails(-5, dist, engine, 1 << 22)            # RP_ERR_TIMEOUT
    rp.rp_debug_faults("clear")
    assert_parity(dist, engine, 2024, None, 0, 1 << 20)


def test_tail_queue_overflow_is_reported():
    rp.rp_debug_faults("tail_cap", 2)            # a 2^20 normal fill has ~270 tail outputs
    msg = _fails(-7, "normal", "pcg64dxsm", 1 << 20)   # RP_ERR_INTERNAL
    assert "device check failed" in msg
    rp.rp_debug_faults("clear")
    assert_parity("normal", "pcg64dxsm", 2024, None, 0, 1 << 20)


def test_continuation_launches():
    """A fill split over launches of two tiles each equals the oracle; one
    that would need more than 64 launches fails cleanly."""
    rp.rp_debug_faults("tile_cap", 2)
    for dist in ("normal", "exp"):
        assert_parity(dist, "xoshiro256pp", 2024, None, 3, 300_000)
    rp.rp_debug_faults("tile_cap", 1)
    msg = _fails(-7, "normal", "xoshiro256pp", 1 << 22)
    assert "continuation" in msg
    rp.rp_debug_faults("clear")
    assert_parity("normal", "xoshiro256pp", 2024, None, 0, 1 << 20)


def test_unknown_fault_kind_is_refused():
    with pytest.raises(rp.RPError) as ei:
        rp.rp_debug_faults(9, 1)
    assert ei.value.code == -2
