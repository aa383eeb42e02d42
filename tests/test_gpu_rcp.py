"""The FP32 reciprocal of the collision (1/s0, the 1/(s0 + mu0/r^2) and
1/(1 + u_r/2r) factors of Eqs. 16-17, and 1/r): a hardware estimate refined
by one Newton-Raphson step.  Against 1/x in FP64 it must stay within one ulp
(faithful rounding) over the arguments the solver meets and well beyond;
the scalar form (boundary kernels) and the paired-lane form (bulk kernels)
must agree bit for bit, so that both kernels round a node alike."""
import numpy as np
import pytest

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


def test_reciprocal_is_faithful_and_lanes_agree(B):
    rng = np.random.default_rng(11)
    x = np.concatenate([
        np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 400_000)),   # wide range
        rng.uniform(0.5, 2.0, 400_000),                            # densities near rho0 = 1
        np.arange(1, 20001) - 0.5, np.arange(1, 20001, dtype=float),  # half-spacing and node radii
        [1.0, 2.0, 0.5, 3.0, 1.0 + 2.0 ** -23, 1.0 - 2.0 ** -24],
    ]).astype(np.float32)
    scalar, paired = B.axlbm_selftest_rcp(x)
    assert np.array_equal(scalar.view(np.uint32), paired.view(np.uint32))
    exact = 1.0 / x.astype(np.float64)
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    err = np.abs(scalar.astype(np.float64) - exact) / ulp
    assert err.max() < 1.0, float(err.max())
    # powers of two are exact
    p2 = np.float32(2.0) ** np.arange(-20, 21, dtype=np.float32)
    s2, _ = B.axlbm_selftest_rcp(p2)
    assert np.array_equal(s2, (1.0 / p2.astype(np.float64)).astype(np.float32))
    # share of results equal to the correctly rounded reciprocal (reported, not bounded)
    rn = (1.0 / x.astype(np.float64)).astype(np.float32)
    assert np.mean(scalar == rn) > 0.9


def test_reciprocal_rejects_bad_arguments(B):
    import ctypes
    L = B.lib()
    out = np.empty(2, dtype=np.float32)
    assert L.axlbm_selftest_rcp(None, 1, out.ctypes.data) == B.EINVAL
    assert L.axlbm_selftest_rcp(out.ctypes.data, 0, out.ctypes.data) == B.EINVAL
