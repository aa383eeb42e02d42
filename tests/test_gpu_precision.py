"""Error of the 16-bit deviation storage modes against the FP64 oracle.

FP16 / BF16 storage keeps f_a - w_a rho0, g_a and h_a - T_ref/4 in 16 bits
and collides in FP32.  Each test runs the same seeded state through the
oracle and the GPU and states the error per macroscopic field, relative to
the field's own scale (rho: to rho0; u_r, u_z, u_theta: to max |u|; T: to the
wall temperature difference).  Bounds follow from the storage precision:
the rounding of a stored deviation of size ~1e-2 is ~1e-2 * 2^-11 (FP16) or
~1e-2 * 2^-8 (BF16) per step, damped by the collision; the bounds below leave
room for the accumulated rounding over the run.
"""

import numpy as np
import pytest

import oracle
from paper_1003_0282_gb300 import inputs as I

from parity_util import record

pytestmark = pytest.mark.gpu

BOUNDS = {  # relative max-norm after 200 steps
    "fp16": {"rho": 2e-4, "u_r": 5e-3, "u_z": 5e-3, "u_theta": 5e-3, "T": 2e-3},
    "bf16": {"rho": 2e-3, "u_r": 5e-2, "u_z": 5e-2, "u_theta": 5e-2, "T": 2e-2},
    "fp32": {"rho": 1e-6, "u_r": 1e-5, "u_z": 1e-5, "u_theta": 1e-5, "T": 1e-5},
}


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import build
    build.build()
    from paper_1003_0282_gb300 import axlbm
    return axlbm


def field_errors(got, want, pb):
    names = ["rho", "u_r", "u_z", "u_theta", "T"]
    uscale = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])), 1e-12)
    scales = {"rho": pb.rho0, "u_r": uscale, "u_z": uscale,
              "u_theta": max(np.max(np.abs(want[3])), 1e-12), "T": 1.0}
    return {n: float(np.max(np.abs(got[q] - want[q])) / scales[n]) for q, n in enumerate(names)}


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_reduced_storage_error_per_field(B, precision):
    pb = I.wheeler_cell(nr=96, re_x=300.0, prandtl=1.0, grashof=3e4)  # swirl + temperature + mixed top
    fields = I.random_fields(pb.nr, pb.nz, seed=17, du=2e-2, duth=2e-2)
    st = oracle.equilibrium(pb, fields)
    dom = B.Domain(pb, precision)
    dom.set_populations(st.f, st.g, st.h, time=0)
    dom.step(200)
    oracle.step(st, 200)
    got = dom.moments(B.RHO | B.UR | B.UZ | B.UTH | B.T)
    errs = field_errors(got, oracle.moments(st), pb)
    dom.close()
    _record(precision, errs)
    for name, bound in BOUNDS[precision].items():
        assert errs[name] <= bound, (name, errs)


def _record(key, value):
    record("precision_errors.json", key, value)


CAVITY_BOUNDS = {"fp32": 1e-5, "fp16": 2e-2, "bf16": 1e-1}  # relative max-norm on u_r, u_z, u_theta


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_reduced_storage_lid_driven_cavity(B, precision):
    """Boundary-driven flow, the intended use of 16-bit storage: a rotating-lid
    cylinder (A = 1.5, Re = 100, 24 x 36 nodes) run for 30000 steps from rest,
    close to steady; velocities against the oracle's."""
    pb = I.rotating_lid_cavity(nr=24, aspect=1.5, re=100.0)
    st = oracle.rest_state(pb)
    dom = B.Domain(pb, precision)
    dom.step(30000)
    oracle.step(st, 30000)
    got = dom.moments(B.RHO | B.UR | B.UZ | B.UTH)
    want = oracle.moments(st)
    dom.close()
    scale = max(np.max(np.abs(want[q])) for q in (1, 2, 3))
    errs = {name: float(np.max(np.abs(got[q] - want[q])) / scale) for q, name in ((1, "u_r"), (2, "u_z"), (3, "u_theta"))}
    _record(f"cavity_{precision}", errs)
    assert max(errs.values()) <= CAVITY_BOUNDS[precision], errs


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_reduced_storage_weak_forcing_is_recorded(B, precision):
    """Known limitation, recorded rather than bounded: in Hagen-Poiseuille flow
    with u_max = 0.01 the per-step force increment of a population (about
    w * 3a = 1.3e-6) is below half a unit in the last place of its 16-bit
    deviation, so round-to-nearest storage loses it and the steady profile
    drifts far from Eq. 55.  The test records the error and the residual."""
    from oracle import analytic as A
    pb = I.hagen_poiseuille(nr=32, nz=8, tau=0.8, umax=0.01)
    dom = B.Domain(pb, precision)
    dom.step(25000)
    uz = dom.moments(B.UZ)[0]
    res, _, _ = dom.residual()
    dom.close()
    nu = (pb.tau - 0.5) / 3
    ua = A.hagen_poiseuille(oracle.node_radii(pb), 32, pb.az0, nu)
    err = float(np.sqrt(np.mean((uz - ua) ** 2)) / np.max(ua))
    _record(f"hagen_poiseuille_{precision}", {"rms_error_rel_umax": err, "residual": res})
    assert np.isfinite(err) and np.isfinite(res)
