"""Batched uneven domains in one persistent launch, against the oracle.

Each domain of a batch must follow exactly the single-domain update: the
tests compare every domain with the FP64 oracle after 1, 2, ... steps, check
that a batch reproduces single-domain runs bit for bit (each node's update
depends only on its own inputs, so packing and tile order cannot change it),
and check the per-domain check-step statistics.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1003_0282_gb300 import inputs as I
from parity_util import POP_TOL, rel_err, seeded_state

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


def mixed_batch():
    """Uneven domains: cavities of several sizes and Reynolds numbers, a
    Wheeler-type cell with temperature, an annulus, a free-surface cell."""
    doms = [
        I.rotating_lid_cavity(nr=70, aspect=1.5, re=300.0),
        I.rotating_lid_cavity(nr=33, aspect=2.5, re=150.0),
        I.wheeler_cell(nr=40, re_x=200.0, prandtl=1.0, grashof=2e4),
        I.rotating_lid_cavity(nr=130, aspect=1.0, re=500.0),
        dataclasses.replace(I.rotating_lid_cavity(nr=20, aspect=3.0, re=100.0), z_hi="free"),
        dataclasses.replace(I.rotating_lid_cavity(nr=25, aspect=1.2, re=100.0), inner="wall", r0=6.0,
                            omega={"inner": 0.002, "hi": 0.004}),
        I.wheeler_cell(nr=17, re_x=150.0, prandtl=5.0, grashof=1e4),
    ]
    return doms


@pytest.mark.parametrize("precision", ["fp32"])
def test_batch_matches_oracle_per_domain(B, precision):
    doms = mixed_batch()
    batch = B.Batch(doms, precision)
    states = []
    for d, pb in enumerate(doms):
        st = seeded_state(pb, 100 + d)
        batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        states.append(st)
    worst = 0.0
    for n in (1, 1, 2, 7, 29):
        batch.step(n)
        for d, pb in enumerate(doms):
            oracle.step(states[d], n)
            f, g, h = batch.get_populations(d)
            errs = [rel_err(f, states[d].f), rel_err(g, states[d].g)]
            if pb.temperature:
                errs.append(rel_err(h, states[d].h))
            worst = max(worst, max(errs))
    assert batch.time == 40
    batch.close()
    assert worst <= POP_TOL[precision], worst


def test_batch_equals_single_domain_runs_bitwise(B):
    doms = mixed_batch()
    batch = B.Batch(doms, "fp32")
    singles = []
    for d, pb in enumerate(doms):
        st = seeded_state(pb, 200 + d)
        batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        dom = B.Domain(pb, "fp32")
        dom.set_populations(st.f, st.g, st.h if pb.temperature else None, time=0)
        singles.append(dom)
    batch.step(13)
    for d, dom in enumerate(singles):
        dom.step(13)
        fb, gb, hb = batch.get_populations(d)
        fs, gs, hs = dom.get_populations()
        assert np.array_equal(fb, fs) and np.array_equal(gb, gs), d
        if hb is not None:
            assert np.array_equal(hb, hs), d
        rb = batch.moments(d, B.RHO | B.UR | B.UZ | B.UTH)
        rs = dom.moments(B.RHO | B.UR | B.UZ | B.UTH)
        assert np.array_equal(rb, rs), d
        dom.close()
    batch.close()


def test_batch_check_statistics_per_domain(B):
    doms = mixed_batch()
    batch = B.Batch(doms, "fp32")
    refs = []
    for d, pb in enumerate(doms):
        st = seeded_state(pb, 300 + d)
        batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        refs.append(st)
    batch.step(11)   # checks the step 10 -> 11: levels 9 and 10
    res = batch.residuals()
    for d, pb in enumerate(doms):
        ref = refs[d]
        oracle.step(ref, 9)
        _, _, sp9 = oracle.stats(ref)
        oracle.step(ref, 1)
        m10, b10, sp10 = oracle.stats(ref)
        assert res[d, 0] == pytest.approx(float(np.max(np.abs(sp10 - sp9))), rel=2e-3, abs=1e-9), d
        assert res[d, 1] == pytest.approx(m10, rel=1e-7), d
        assert res[d, 2] == pytest.approx(b10, rel=1e-3, abs=1e-9), d
    batch.step(2)    # an even number of steps: checks ending on an even level use no ring values
    assert np.all(np.isfinite(batch.residuals()))
    batch.close()


def test_batch_fields_io_and_parity_rule(B):
    doms = mixed_batch()[:3]
    batch = B.Batch(doms, "fp32")
    fields = I.random_fields(doms[2].nr, doms[2].nz, seed=9)
    batch.set_fields(2, fields)
    want = oracle.equilibrium(doms[2], fields)
    f, g, h = batch.get_populations(2)
    assert rel_err(f, want.f) <= 1e-6 and rel_err(g, want.g) <= 1e-6 and rel_err(h, want.h) <= 1e-6
    batch.step(1)
    with pytest.raises(B.AxlbmError) as ei:
        batch.set_fields(0, I.random_fields(doms[0].nr, doms[0].nz, seed=1))
    assert ei.value.status == B.EINVAL
    batch.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_full_sweep_sampled_domains(B, precision):
    """The uneven sweep (256 rotating-lid cavities with N_r in [64, 256] and
    64 Wheeler-type 128 x 128 cells, about 17.6 M nodes) in one batch; a few
    domains are compared whole with the oracle after 6 steps from a seeded
    state, every domain's mass budget is checked."""
    doms = I.batch_sweep()
    batch = B.Batch(doms, precision)
    picks = [0, 7, 255, 256, 300, 319]
    small = sorted(set(sorted(picks, key=lambda d: doms[d].cells)[:4]) | {300})  # 300: a Wheeler cell (h)
    states = {}
    for d in small:
        st = seeded_state(doms[d], 500 + d)
        batch.set_populations(d, st.f, st.g, st.h if doms[d].temperature else None)
        states[d] = st
    batch.step(5)
    r5 = batch.residuals()
    batch.step(1)
    r6 = batch.residuals()
    tol = POP_TOL.get(precision, 5e-3)
    for d in small:
        oracle.step(states[d], 6)
        f, g, h = batch.get_populations(d)
        assert rel_err(f, states[d].f) <= tol and rel_err(g, states[d].g) <= max(tol, 1e-4 if precision == "fp16" else tol), d
        if doms[d].temperature:
            assert rel_err(h, states[d].h) <= tol, d
    assert any(doms[d].temperature for d in small)
    # mass budget M(6) = M(5) - B(5) in every domain (storage rounding only)
    mtol = 1e-9 if precision == "fp32" else 1e-5
    assert np.all(np.abs(r6[:, 1] - (r5[:, 1] - r5[:, 2])) <= mtol * np.abs(r5[:, 1]))
    batch.close()


def test_batch_packed_fields_match_per_domain_calls(B):
    doms = mixed_batch()
    batch = B.Batch(doms, "fp32")
    packed = np.concatenate([I.random_fields(pb.nr, pb.nz, seed=40 + d).ravel() for d, pb in enumerate(doms)])
    batch.set_fields_all(packed)
    off = 0
    for d, pb in enumerate(doms):
        want = oracle.equilibrium(pb, packed[off:off + 5 * pb.cells].reshape(5, pb.nz, pb.nr))
        f, g, _ = batch.get_populations(d)
        assert rel_err(f, want.f) <= 1e-6 and rel_err(g, want.g) <= 1e-6, d
        off += 5 * pb.cells
    batch.step(3)
    mask = B.RHO | B.UR | B.UZ | B.UTH
    allm = np.empty(sum(4 * pb.cells for pb in doms), dtype=np.float32)
    batch.moments_all(mask, allm)
    off = 0
    for d, pb in enumerate(doms):
        one = batch.moments(d, mask, dtype=np.float32)
        assert np.array_equal(allm[off:off + 4 * pb.cells].reshape(4, pb.nz, pb.nr), one), d
        off += 4 * pb.cells
    batch.close()


def test_batch_async_host_io_matches_the_synchronous_calls(B):
    """Fields in and moments out through the copy stream, three rounds queued
    before one sync (the two staging buffers each way are reused), against the
    same sequence of synchronous calls, bit for bit: FP32 from pinned memory,
    FP64 from pageable memory, results into pinned and pageable memory."""
    import torch

    doms = mixed_batch()
    cells = sum(pb.cells for pb in doms)
    mask = B.RHO | B.UR | B.UZ
    fin = []
    for n in range(3):
        a = np.concatenate([I.random_fields(pb.nr, pb.nz, seed=90 + 7 * n + d).ravel() for d, pb in enumerate(doms)])
        fin.append(a if n == 1 else torch.from_numpy(a.astype(np.float32)).pin_memory())
    want = []
    ref = B.Batch(doms, "fp32")
    for n in range(3):
        ref.set_fields_all(fin[n])
        ref.step(4)
        out = np.empty(3 * cells, dtype=np.float32)
        ref.moments_all(mask, out)
        want.append(out)
    ref.close()
    batch = B.Batch(doms, "fp32")
    outs = [torch.empty(3 * cells, dtype=torch.float32).pin_memory(), np.empty(3 * cells, dtype=np.float32),
            torch.empty(3 * cells, dtype=torch.float32).pin_memory()]
    for n in range(3):
        batch.set_fields_all_async(fin[n])
        batch.step(4)
        batch.moments_all_async(mask, outs[n])
    batch.sync()
    for n in range(3):
        got = outs[n].numpy() if isinstance(outs[n], torch.Tensor) else outs[n]
        assert np.array_equal(got, want[n]), n
    with pytest.raises(ValueError):
        batch.moments_all_async(mask, np.empty((3, cells), dtype=np.float32)[:, ::2])
    batch.step(1)
    with pytest.raises(B.AxlbmError):
        batch.set_fields_all_async(np.zeros(5 * cells))  # fields are set at an even level
    batch.close()


def test_batch_mixes_bgk_and_mrt_domains(B):
    doms = mixed_batch()
    doms = [dataclasses.replace(pb, collision="mrt") if i % 2 else pb for i, pb in enumerate(doms)]
    batch = B.Batch(doms, "fp32")
    states = []
    for d, pb in enumerate(doms):
        st = seeded_state(pb, 700 + d)
        batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        states.append(st)
    batch.step(9)
    for d, pb in enumerate(doms):
        oracle.step(states[d], 9)
        f, g, h = batch.get_populations(d)
        assert rel_err(f, states[d].f) <= POP_TOL["fp32"], (d, pb.collision)
        assert rel_err(g, states[d].g) <= POP_TOL["fp32"], (d, pb.collision)
    batch.close()


def test_batch_with_node_on_axis_and_wet_wall_domains(B):
    """Domains with a node on the axis (Sec. IV A) and with wet walls (Sec.
    IV B) beside plain ones, BGK and MRT, against the oracle; the mirror and
    rebuild passes run for those domains only."""
    doms = mixed_batch()[:4] + [
        dataclasses.replace(I.rotating_lid_cavity(nr=45, aspect=1.4, re=200.0), inner="axis_node"),
        dataclasses.replace(I.wheeler_cell(nr=38, re_x=200.0, prandtl=1.0, grashof=2e4), inner="axis_node",
                            collision="mrt"),
        dataclasses.replace(I.rotating_lid_cavity(nr=30, aspect=2.0, re=150.0), inner="axis_node", z_hi="free"),
        # wet walls (non-equilibrium extrapolation)
        dataclasses.replace(I.rotating_lid_cavity(nr=41, aspect=1.5, re=300.0), inner="axis_node", outer="nee",
                            z_lo="nee", z_hi="nee", collision="mrt"),
        dataclasses.replace(I.wheeler_cell(nr=36, re_x=150.0, prandtl=1.0, grashof=1e4), outer="nee", z_lo="nee"),
    ]
    batch = B.Batch(doms, "fp32")
    states = []
    for d, pb in enumerate(doms):
        st = seeded_state(pb, 800 + d)
        batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        states.append(st)
    for n in (1, 1, 5):
        batch.step(n)
        for d, pb in enumerate(doms):
            oracle.step(states[d], n)
            f, g, h = batch.get_populations(d)
            assert rel_err(f, states[d].f) <= POP_TOL["fp32"], (d, pb.inner)
            assert rel_err(g, states[d].g) <= POP_TOL["fp32"], (d, pb.inner)
            if pb.temperature:
                assert rel_err(h, states[d].h) <= POP_TOL["fp32"], (d, pb.inner)
    batch.close()


def test_kernel_times_split_by_parity(B):
    """The per-parity bulk totals add up to the overall ones; an even number
    of steps from an even level times as many even as odd launches, and the
    odd launches count the interior nodes only."""
    doms = mixed_batch()
    batch = B.Batch(doms, "fp32")
    B.axlbm_batch_kernel_timing(batch.handle, True)
    batch.step(10)
    n, ms, by, _ = B.axlbm_batch_kernel_times(batch.handle)
    n2, ms2, by2 = B.axlbm_batch_kernel_times_by_parity(batch.handle)
    assert n2 == [5, 5] and n == 10
    assert abs(sum(ms2) - ms) <= 1e-9 * max(ms, 1.0) and min(ms2) > 0.0
    assert abs(sum(by2) - by) <= 1e-6 * by
    interior = sum((pb.nr - 2) * (pb.nz - 2) for pb in doms)
    assert by2[1] < by2[0] and by2[1] >= 5 * interior * 2 * 13 * 4
    B.axlbm_batch_kernel_timing(batch.handle, True)  # re-enabling clears the totals
    assert B.axlbm_batch_kernel_times_by_parity(batch.handle)[0] == [0, 0]
    batch.close()


def test_results_do_not_depend_on_the_tile_shape(B):
    """Every bulk tile shape gives the same populations and residuals bit for
    bit (each node's update depends only on its own inputs), including a
    switch of shape between calls; the mass and budget sums differ only by
    their summation order.  An unknown shape is refused."""
    doms = mixed_batch()
    runs = []
    # (even-step shape, odd-step shape) per call
    for shapes in ([((4, 128), (4, 128))] * 2, [((8, 64), (8, 64))] * 2, [((8, 64), (4, 128)), ((4, 128), (8, 64))]):
        batch = B.Batch(doms, "fp32")
        for d, pb in enumerate(doms):
            st = seeded_state(pb, seed=70 + d)
            batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        for even, odd in shapes:
            if even == odd:
                batch.tile_shape = even
            else:
                batch.tile_shapes = (even, odd)
            assert batch.tile_shapes == (even, odd) and batch.tile_shape == even
            batch.step(3)
        for bad in ((4, 32), (2, 128)):
            with pytest.raises(B.AxlbmError):
                batch.tile_shape = bad
        with pytest.raises(B.AxlbmError):
            batch.tile_shapes = ((4, 128), (4, 64))
        runs.append(([batch.get_populations(d) for d in range(len(doms))], batch.residuals()))
        batch.close()
    pops0, res0 = runs[0]
    for pops, res in runs[1:]:
        assert np.array_equal(res[:, 0], res0[:, 0])
        assert np.all(np.abs(res[:, 1:] - res0[:, 1:]) <= 1e-9 * res0[:, 1:2])
        for d in range(len(doms)):
            for x, y in zip(pops[d], pops0[d]):
                assert (x is None and y is None) or np.array_equal(x, y), d


def test_fp16_tile_shapes_give_the_same_state(B):
    """With 16-bit storage the bulk kernel also runs 8 x 128 tiles (each
    computing thread updates two node pairs of its column): the populations
    and residuals equal those of the 512-node tiles bit for bit, in every
    combination of even- and odd-step shapes."""
    doms = mixed_batch()
    runs = []
    for shapes in (((4, 128), (4, 128)), ((8, 128), (8, 128)), ((8, 128), (4, 128)), ((8, 64), (8, 128))):
        batch = B.Batch(doms, "fp16")
        for d, pb in enumerate(doms):
            st = seeded_state(pb, seed=170 + d)
            batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        batch.tile_shapes = shapes
        assert batch.tile_shapes == shapes
        batch.step(7)
        runs.append(([batch.get_populations(d) for d in range(len(doms))], batch.residuals()))
        batch.close()
    pops0, res0 = runs[0]
    for pops, res in runs[1:]:
        assert np.array_equal(res[:, 0], res0[:, 0])
        assert np.all(np.abs(res[:, 1:] - res0[:, 1:]) <= 1e-9 * res0[:, 1:2])  # mass and budget: summation order
        for d in range(len(doms)):
            for x, y in zip(pops[d], pops0[d]):
                assert (x is None and y is None) or np.array_equal(x, y), d
    fp32 = B.Batch(doms, "fp32")
    with pytest.raises(B.AxlbmError):
        fp32.tile_shape = (8, 128)  # its stages would not fit two CTAs per SM with FP32 storage
    fp32.close()


def test_graph_replay_matches_direct_launches(B):
    """Runs of plain steps replayed from captured CUDA graphs give the same
    populations and check values bit for bit as launching every kernel, from
    an odd start, across a tile-shape change (recapture) and with wet-wall
    and node-on-axis domains in the batch (their passes are in the graph)."""
    doms = mixed_batch() + [
        dataclasses.replace(I.wheeler_cell(nr=21, re_x=200.0, prandtl=1.0, grashof=1e4), inner="axis_node"),
        dataclasses.replace(I.rotating_lid_cavity(nr=17, aspect=1.5, re=200.0), outer="nee", z_lo="nee"),
    ]
    out = []
    for graphs in (True, False):
        batch = B.Batch(doms, "fp32")
        batch.use_graphs(graphs)
        for d, pb in enumerate(doms):
            st = seeded_state(pb, seed=90 + d)
            batch.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
        batch.step(1)
        for n in (23, 30):
            batch.step(n)
        batch.tile_shape = (8, 64) if batch.tile_shape == (4, 128) else (4, 128)
        batch.step(21)  # sizes the new shape's kernels if no tuning run did
        batch.step(21)
        caps, launches = batch.graph_stats()
        if graphs:
            assert caps == 2 and launches >= 3, (caps, launches)
        else:
            assert caps == 0 and launches == 0
        out.append(([batch.get_populations(d) for d in range(len(doms))], batch.residuals(), batch.time))
        batch.close()
    (p0, r0, t0), (p1, r1, t1) = out
    assert t0 == t1 == 96
    assert np.array_equal(r0, r1)
    for d in range(len(doms)):
        for x, y in zip(p0[d], p1[d]):
            assert (x is None and y is None) or np.array_equal(x, y), d


def test_repacked_domains_continue_bit_for_bit(B):
    """Domains copied into a smaller batch at the same even time level
    (axlbm_batch_set_time + axlbm_batch_copy_domain) continue exactly as in the
    original batch -- including a pipe with an oscillating axial force, whose
    a(t) follows the time level; the check sums agree up to their summation
    order.  Copies between different grids or storage, and odd levels, are
    refused."""
    pipe = I.Problem(nr=20, nz=12, tau=0.8, inner="axis", z_lo="periodic", z_hi="periodic", swirl=True,
                     az0=2e-5, omega_t=0.01)
    doms = mixed_batch() + [pipe]
    full = B.Batch(doms, "fp32")
    for d, pb in enumerate(doms):
        st = seeded_state(pb, seed=110 + d)
        full.set_populations(d, st.f, st.g, st.h if pb.temperature else None)
    full.step(20)
    keep = [1, 3, len(doms) - 1, 5, 2]
    sub = B.Batch([doms[d] for d in keep], "fp32")
    with pytest.raises(B.AxlbmError):
        sub.copy_domain(0, full, keep[0])  # different time levels
    sub.set_time(full.time)
    assert sub.time == full.time == 20
    for k, d in enumerate(keep):
        sub.copy_domain(k, full, d)
    with pytest.raises(B.AxlbmError):
        sub.copy_domain(0, full, 0)  # another grid
    full.step(31)
    sub.step(31)
    rf, rs = full.residuals(), sub.residuals()
    for k, d in enumerate(keep):
        for x, y in zip(sub.get_populations(k), full.get_populations(d)):
            assert (x is None and y is None) or np.array_equal(x, y), d
        assert rs[k, 0] == rf[d, 0]
        assert np.all(np.abs(rs[k, 1:] - rf[d, 1:]) <= 1e-9 * rf[d, 1])
    with pytest.raises(B.AxlbmError):
        sub.set_time(52)  # the batch is at an odd level
    half = B.Batch([doms[1]], "fp16")
    with pytest.raises(B.AxlbmError):
        half.copy_domain(0, full, 1)  # another storage
    half.close()
    sub.close()
    full.close()
