"""Device self-tests that run before any parity test: the tensor-core operand layout and
the bounded-wait (watchdog) path."""
import numpy as np
import pytest

from paper_1805_11125_gb300 import bx

pytestmark = pytest.mark.gpu


def test_tensor_core_layout_selftest():
    """128x32 by 16x32 product through the TF32 hi/lo split, UMMA layouts, tcgen05.mma and
    tensor-memory read-back; TF32x3 keeps ~2^-21 relative accuracy per product."""
    err = bx.bx_selftest_tensor_core()
    assert err < 1e-5, err


def test_watchdog_times_out_and_context_survives():
    """A wait on a barrier that nothing arrives on ends after its budget with BX_ETIMEOUT;
    the CUDA context keeps working."""
    assert bx.bx_selftest_watchdog(0.02) == bx.BX_ETIMEOUT
    assert bx.bx_selftest_tensor_core() < 1e-5
