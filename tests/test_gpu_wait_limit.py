"""The error path of the bounded device waits.

Every wait of the bulk kernels on a TMA copy gives up after a cycle budget
and the step then reports AXLBM_ETIMEOUT instead of hanging the GPU.  In a
correct run that path never executes, so the library's self-test runs it on
a barrier that nothing completes, with a budget of about a millisecond: all
32 threads must give up, the warp must raise the error word, and the device
must stay usable afterwards.  Nothing here faults or hangs a GPU.
"""
import time

import numpy as np
import pytest

from paper_1003_0282_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import build
    build.build()
    from paper_1003_0282_gb300 import axlbm
    return axlbm


def test_bounded_wait_gives_up_and_reports(B):
    t0 = time.perf_counter()
    gave_up, err = B.axlbm_selftest_bounded_wait(2_000_000)  # ~1 ms at 2 GHz
    assert time.perf_counter() - t0 < 10.0
    assert gave_up == 32 and err == 1
    # the context is still usable: a small domain steps normally afterwards
    pb = I.rotating_lid_cavity(nr=16, aspect=1.5, re=100.0)
    dom = B.Domain(pb, "fp32")
    dom.step(4)
    res, mass, _ = dom.residual()
    assert np.isfinite(res) and np.isfinite(mass)
    dom.close()


def test_bounded_wait_budget_is_checked(B):
    for bad in (0, 999, 4_000_000_001):
        with pytest.raises(B.AxlbmError):
            B.axlbm_selftest_bounded_wait(bad)
