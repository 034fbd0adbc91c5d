"""Failure detection without a GPU fault: the bounded wait that guards every
TMA stage of the forward gives up after its limit, the kernel records
PA_ERR_TIMEOUT in the device error word, the host reads it, and the context
keeps working (a forward afterwards still matches the FP64 oracle)."""
import numpy as np
import pytest

import oracle
import pa_inputs
from gpu_common import TRACE_TOL, dev_pad, geometry, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def test_bounded_wait_times_out_and_the_context_survives(pa):
    from paper_2412_03898_gb300 import _lib
    pa.device_error()  # start from a clear error word
    pa.selftest_bounded_wait(2_000_000)  # 2 ms on an mbarrier nothing completes
    with pytest.raises(pa.PAError) as e:
        pa.device_error()
    assert e.value.status == _lib.PA_ERR_TIMEOUT
    pa.device_error()  # reading cleared it
    sc = pa_inputs.small_scene(seed=8, n_balls=257, n_sensors=9, n_samples=512)
    y = pa.forward(geometry(sc), dev_pad(sc.balls)[None], sc.n_balls)
    pa.device_error()
    y_o, _ = oracle.forward(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL


def test_selftest_limit_is_bounded(pa):
    with pytest.raises(pa.PAError):
        pa.selftest_bounded_wait(10)  # below 1 us
    with pytest.raises(pa.PAError):
        pa.selftest_bounded_wait(5_000_000_000)  # above 1 s
