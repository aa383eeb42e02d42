"""z-slab decomposition on the GPU: one domain cut across z into slabs (two
or three handles on this GPU, cut faces AXLBM_Z_HALO, exchanged after every
step through device buffers) against the undivided domain, from the same
seeded state, after 1, 2 and 101 steps: periodic ends (the pipes of
Sec. IV A) and closed ends, with g and h, BGK and MRT, FP64 and FP32.

The slab run must give the undivided run's populations.  The rows next to a
cut are updated by the boundary-ring kernel (one node per thread) instead of
the bulk kernel (in FP32 two nodes per thread with paired FP32
instructions); with BGK in FP64 the two round alike and the runs match bit
for bit, with MRT in FP64 the compiler fuses a few multiply-adds of the
moment-space collision differently in the two kernels (held to 1e-13), and
FP32 is held to 1e-6 of the population scale.  Check values: the largest
slab residual is the domain's, the slab masses and budgets add up to the
domain's.
"""
import dataclasses

import numpy as np
import pytest

from paper_1003_0282_gb300 import inputs as I
from parity_util import problem, rel_err, seeded_state, upload

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


CASES = [("pipe", 2, "bgk"), ("pipe", 3, "mrt"), ("closed", 2, "bgk"), ("crystal", 3, "mrt"),
         ("annulus-pipe", 2, "bgk")]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mix,nslabs,collision", CASES)
def test_slabs_equal_the_undivided_domain(B, mix, nslabs, collision, precision):
    from paper_1003_0282_gb300 import slab as SL

    pb = problem(150, 61, mix, collision=collision)
    st = seeded_state(pb, 71)
    whole = B.Domain(pb, precision)
    upload(whole, st)
    slabs = SL.LocalSlabs(pb, nslabs, precision)
    slabs.set_populations(st.f, st.g, st.h, time=st.t)
    tol = (0.0 if collision == "bgk" else 1e-13) if precision == "fp64" else 1e-6
    for n in (1, 1, 99):
        for _ in range(n):
            whole.step(1)  # a check step every step, as the slabs take
        slabs.step(n)
        assert slabs.time == whole.time
        fw, gw, hw = whole.get_populations()
        fs, gs, hs = slabs.get_populations()
        for got, want in ((fs, fw), (gs, gw), (hs, hw)):
            if tol == 0.0:
                assert np.array_equal(got, want), (mix, n)
            else:
                assert rel_err(got, want) <= tol, (mix, n, rel_err(got, want))
        rw, mw, bw = whole.residual()
        rs, ms, bs = slabs.residual()
        assert rs == pytest.approx(rw, rel=1e-12 if precision == "fp64" else 1e-3, abs=1e-15)
        assert ms == pytest.approx(mw, rel=1e-13 if precision == "fp64" else 1e-7)
        assert bs == pytest.approx(bw, rel=1e-9 if precision == "fp64" else 1e-3, abs=1e-12)
    mask = B.RHO | B.UR | B.UZ | B.UTH | B.T
    assert rel_err(slabs.moments(mask), whole.moments(mask)) <= (1e-13 if precision == "fp64" else 1e-5)
    whole.close()
    slabs.close()


def test_cut_faces_enforce_the_exchange(B):
    from paper_1003_0282_gb300 import slab as SL

    pb = problem(40, 20, "pipe")
    slabs = SL.LocalSlabs(pb, 2, "fp64")
    d0 = slabs.doms[0]
    with pytest.raises(B.AxlbmError):
        d0.step(2)                      # one step per call
    buf = np.empty(d0.halo_bytes(), np.uint8)
    with pytest.raises(B.AxlbmError):
        d0.halo_send(B.FACE_LO, buf)    # nothing to exchange yet
    d0.step(1)
    with pytest.raises(B.AxlbmError):
        d0.step(1)                      # the cut faces have not received their messages
    with pytest.raises(B.AxlbmError):
        d0.halo_send(B.FACE_INNER, buf)
    assert d0.halo_bytes() == (3 + 1 + 1) * 40 * 8
    slabs.close()
    # cut faces are for the half-spacing axis or an inner wall, bounce-back outer wall, no wet walls
    for bad in (dict(inner="axis_node"), dict(outer="nee")):
        with pytest.raises(B.AxlbmError):
            B.Domain(dataclasses.replace(problem(40, 20, "pipe"), z_lo="halo", z_hi="halo", **bad), "fp64")
    with pytest.raises(B.AxlbmError):
        B.Batch([dataclasses.replace(I.rotating_lid_cavity(nr=40, aspect=1.0, re=100.0), z_lo="halo")], "fp32")


def test_slab_pipe_hagen_poiseuille_profile(B):
    """Hagen-Poiseuille (Eq. 55) through three FP64 slabs of a periodic pipe:
    the same profile as the undivided pipe, bit for bit, after 3000 steps."""
    from paper_1003_0282_gb300 import slab as SL

    pb = I.hagen_poiseuille(nr=32, nz=12, tau=0.8, umax=0.01)
    whole = B.Domain(pb, "fp64")
    slabs = SL.LocalSlabs(pb, 3, "fp64")
    for _ in range(3000):
        whole.step(1)
    slabs.step(3000)
    assert np.array_equal(slabs.moments(B.UZ), whole.moments(B.UZ))
    whole.close()
    slabs.close()
