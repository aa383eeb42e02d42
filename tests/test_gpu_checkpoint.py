"""Checkpoint and resume: axlbm_save / axlbm_load and axlbm_batch_save /
axlbm_batch_load.

A run saved at any level (even or odd AA parity) and resumed in a fresh
handle -- one that has run and captured its step graphs before the load --
continues bit for bit as the uninterrupted run: populations, time level and
check values.  The pipe carries an oscillating axial force, so a(t) has to
come back with the state, and FP64 storage shows that the populations are
not passed through a conversion (axlbm_get/set_populations add and remove
the weights in FP64, which is not exact).  Checkpoints of another grid,
storage or kind, corrupted or truncated ones, are refused and leave the
state unchanged.
"""
import dataclasses

import numpy as np
import pytest

from paper_1003_0282_gb300 import inputs as I
from parity_util import seeded_state

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


# Periodic pipe with swirl and the oscillating axial force a(t) = az0 cos(omega_t t).
PIPE = I.Problem(nr=20, nz=12, tau=0.8, inner="axis", z_lo="periodic", z_hi="periodic", swirl=True,
                 az0=2e-5, omega_t=0.01)
# Wheeler-type cell with temperature and a node on the axis.
CELL = dataclasses.replace(I.wheeler_cell(nr=19, re_x=150.0, prandtl=1.0, grashof=1e4), inner="axis_node")


def same(p, q):
    for x, y in zip(p, q):
        assert (x is None and y is None) or np.array_equal(x, y)


def start(dom, pb, seed):
    st = seeded_state(pb, seed)
    dom.set_populations(st.f, st.g if pb.swirl else None, st.h if pb.temperature else None, time=0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("first", [17, 20])
@pytest.mark.parametrize("name", ["pipe", "cell"])
def test_domain_resumes_bit_for_bit(B, name, first, precision):
    pb = PIPE if name == "pipe" else CELL
    a = B.Domain(pb, precision)
    start(a, pb, seed=3)
    a.step(first)
    ck = a.save()
    info = B.checkpoint_info(ck)
    assert (info["kind"], info["time"], info["parity"]) == ("domain", first, first % 2)
    assert info["state_bytes"] == ck.size - 64 == B.axlbm_state_bytes(a.grid)
    a.step(25)
    b = B.Domain(pb, precision)
    start(b, pb, seed=4)
    b.step(21)  # another state, step graphs captured
    b.load(ck)
    assert b.time == first
    b.step(25)
    assert a.time == b.time == first + 25
    assert a.residual() == b.residual()
    same(a.get_populations(), b.get_populations())
    # rewinding the original handle repeats the continuation
    a.load(ck)
    a.step(25)
    assert a.residual() == b.residual()
    same(a.get_populations(), b.get_populations())
    a.close()
    b.close()


def test_domain_refuses_foreign_checkpoints(B):
    a = B.Domain(PIPE, "fp32")
    start(a, PIPE, seed=7)
    a.step(5)
    ck = a.save()
    assert ck.size == 64 + B.axlbm_state_bytes(a.grid) and bytes(ck[:7]) == b"AXLBMCK"
    other = B.Domain(dataclasses.replace(PIPE, nz=13), "fp32")
    other.step(3)
    before, t0 = other.get_populations(), other.time
    junk = ck.copy()
    junk[0] ^= 1
    for bad in (ck, ck[:-1], ck[:64], ck[:10], junk):  # other grid; truncated; bad magic
        with pytest.raises(B.AxlbmError) as ei:
            other.load(bad)
        assert ei.value.status == B.EINVAL
    assert other.time == t0
    same(other.get_populations(), before)
    for bad in (ck[:-1], junk):
        with pytest.raises(B.AxlbmError):
            a.load(bad)
    half = B.Domain(PIPE, "fp16")
    with pytest.raises(B.AxlbmError):
        half.load(ck)  # other storage
    batch = B.Batch([PIPE], "fp32")
    with pytest.raises(B.AxlbmError):
        batch.load(ck)  # a domain's checkpoint
    with pytest.raises(B.AxlbmError):
        a.load(batch.save())  # a batch's checkpoint
    a.step(2)
    assert a.time == 7
    for h in (a, other, half, batch):
        h.close()


def batch_domains():
    return [
        I.rotating_lid_cavity(nr=33, aspect=1.5, re=150.0),
        dataclasses.replace(I.rotating_lid_cavity(nr=24, aspect=1.0, re=100.0), outer="nee", z_lo="nee"),
        I.wheeler_cell(nr=21, re_x=200.0, prandtl=1.0, grashof=1e4),
        CELL,
        PIPE,
    ]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_batch_resumes_bit_for_bit(B, precision):
    doms = batch_domains()
    a = B.Batch(doms, precision)
    for d, pb in enumerate(doms):
        st = seeded_state(pb, seed=130 + d)
        a.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
    a.step(21)
    ck = a.save()
    info = B.checkpoint_info(ck)
    assert (info["kind"], info["time"], info["parity"]) == ("batch", 21, 1)
    a.step(30)
    b = B.Batch(doms, precision)
    b.step(22)  # another state, step graphs captured
    b.load(ck)
    assert b.time == 21
    b.step(30)
    assert a.time == b.time == 51
    ra, rb = a.residuals(), b.residuals()
    assert np.array_equal(ra[:, 0], rb[:, 0])
    assert np.all(np.abs(ra[:, 1:] - rb[:, 1:]) <= 1e-9 * np.abs(ra[:, 1:2]))
    for d in range(len(doms)):
        for x, y in zip(a.get_populations(d), b.get_populations(d)):
            assert (x is None and y is None) or np.array_equal(x, y), d
    fewer = B.Batch(doms[:-1], precision)
    with pytest.raises(B.AxlbmError) as ei:
        fewer.load(ck)  # another domain list
    assert ei.value.status == B.EINVAL
    with pytest.raises(B.AxlbmError):
        b.load(ck[:-8])
    for h in (a, b, fewer):
        h.close()
