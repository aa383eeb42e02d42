"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every test here runs on a GPU.  Inputs are seeded and built on the oracle
side; the CUDA library receives them through axlbm_set_populations /
axlbm_set_fields and is compared element by element with the oracle after
1, 2, ... steps (covering both AA parities) on grids that span several
thread-block tiles with ragged tails, under every boundary mix, with and
without the swirl and temperature distributions.

Tolerances (relative max-norm): FP64 1e-10, FP32 1e-5 on populations; the
macroscopic fields are checked against the same bounds scaled by their own
magnitude.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as A
from paper_1003_0282_gb300 import inputs as I
from parity_util import (BOUNDARY_MIXES, POP_TOL, compare_populations, problem, record, rel_err, seeded_state,
                         upload, window_oracle)

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


def run_and_compare(B, pb, precision, schedule, seed=11):
    st = seeded_state(pb, seed)
    dom = B.Domain(pb, precision)
    upload(dom, st)
    worst = {}
    for n in schedule:
        oracle.step(st, n)
        dom.step(n)
        assert dom.time == st.t
        errs = compare_populations(dom, st)
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    dom.close()
    return worst, st


@pytest.mark.parametrize("mix", sorted(BOUNDARY_MIXES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_parity_all_boundaries(B, mix, precision):
    pb = problem(150, 37, mix)  # two 128-wide tiles in r, 19 rows of tiles in z, ragged tails
    worst, _ = run_and_compare(B, pb, precision, [1, 1, 2, 7, 29])
    tol = POP_TOL[precision]
    assert all(v <= tol for v in worst.values()), worst


@pytest.mark.parametrize("mix", sorted(BOUNDARY_MIXES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_parity_mrt(B, mix, precision):
    """The MRT collision (Sec. III B) under every boundary mix, default and
    explicit rates."""
    pb = problem(150, 37, mix, collision="mrt", tau=0.62, s_eps=1.3, s_q=1.1)
    worst, _ = run_and_compare(B, pb, precision, [1, 1, 2, 17])
    assert all(v <= POP_TOL[precision] for v in worst.values()), worst
    pb = problem(61, 23, mix, collision="mrt", tau=0.55)
    worst, _ = run_and_compare(B, pb, precision, [1, 6])
    assert all(v <= POP_TOL[precision] for v in worst.values()), worst


@pytest.mark.parametrize("swirl,temp", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_parity_distribution_sets(B, swirl, temp, precision):
    pb = problem(97, 45, "closed", swirl=swirl, temperature=temp)
    worst, _ = run_and_compare(B, pb, precision, [1, 4, 51])
    assert all(v <= POP_TOL[precision] for v in worst.values()), worst


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (5, 1), (2, 2), (2, 7), (7, 2), (3, 3), (33, 3)])
@pytest.mark.parametrize("mix", ["pipe", "closed", "crystal", "annulus-mixed"])
def test_degenerate_shapes(B, shape, mix):
    nr, nz = shape
    pb = problem(nr, nz, mix)
    worst, _ = run_and_compare(B, pb, "fp64", [1, 1, 3, 10])
    assert all(v <= 1e-10 for v in worst.values()), worst


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_moments_residual_mass_budget(B, precision):
    pb = problem(70, 41, "crystal")
    st = seeded_state(pb, 21)
    dom = B.Domain(pb, precision)
    upload(dom, st)
    oracle.step(st, 12)
    dom.step(12)  # even layout afterwards; the loop below also reads the odd one
    for extra in (0, 1):
        if extra:
            oracle.step(st, 1)
            dom.step(1)
        want = oracle.moments(st)
        got = dom.moments(B.RHO | B.UR | B.UZ | B.UTH | B.T)
        tol = POP_TOL[precision]
        assert np.max(np.abs(got[0] - want[0])) <= tol * pb.rho0
        for q in range(1, 5):
            assert rel_err(got[q], want[q]) <= 10 * tol, q
        got32 = dom.moments(B.UZ | B.T, dtype=np.float32)
        assert rel_err(got32[0].astype(np.float64), want[2]) <= max(10 * tol, 1e-6)
    # The last call (n = 1) checked the step 12 -> 13: the Eq. 57 residual between
    # the pre-collision levels 11 and 12, and mass / budget of level 12.
    res, mass, budget = dom.residual()
    ref = seeded_state(pb, 21)
    oracle.step(ref, 11)
    _, _, sp11 = oracle.stats(ref)
    oracle.step(ref, 1)
    m12, b12, sp12 = oracle.stats(ref)
    want_res = float(np.max(np.abs(sp12 - sp11)))
    fp64 = precision == "fp64"
    assert res == pytest.approx(want_res, rel=1e-9 if fp64 else 2e-3, abs=1e-13)
    assert mass == pytest.approx(m12, rel=1e-12 if fp64 else 1e-7)
    assert budget == pytest.approx(b12, rel=1e-9 if fp64 else 1e-3, abs=1e-12 if fp64 else 1e-9)
    dom.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [3, 4, 21])
def test_residual_over_two_levels(B, precision, n):
    """With residual lag 2 a call of n steps from level t0 records
    max |s(t0 + n - 1) - s(t0 + n - 3)| / 2 (s = sqrt(u_r^2 + u_z^2), Eq. 57
    measured across two levels) and the mass and budget of level t0 + n - 1;
    the single domain and a batch holding the same domain agree with the
    oracle, from both AA parities."""
    pb = problem(70, 41, "crystal")
    for t0 in (6, 7):
        st = seeded_state(pb, 23)
        dom = B.Domain(pb, precision)
        upload(dom, st)
        dom.step(t0)
        dom.set_residual_lag(2)
        dom.step(n)
        res, mass, budget = dom.residual()
        dom.close()
        oracle.step(st, t0 + n - 3)
        _, _, sp_a = oracle.stats(st)
        oracle.step(st, 2)
        m_b, b_b, sp_b = oracle.stats(st)
        want = float(np.max(np.abs(sp_b - sp_a))) / 2
        fp64 = precision == "fp64"
        assert res == pytest.approx(want, rel=1e-9 if fp64 else 2e-3, abs=1e-13), (t0, n)
        assert mass == pytest.approx(m_b, rel=1e-12 if fp64 else 1e-7)
        assert budget == pytest.approx(b_b, rel=1e-9 if fp64 else 1e-3, abs=1e-12 if fp64 else 1e-9)
        if precision == "fp32":
            batch = B.Batch([pb], "fp32")
            st0 = seeded_state(pb, 23)
            batch.set_populations(0, st0.f, st0.g, st0.h)
            batch.step(t0)
            batch.set_residual_lag(2)
            batch.step(n)
            r = batch.residuals()
            batch.close()
            assert r[0, 0] == pytest.approx(want, rel=2e-3, abs=1e-13), (t0, n)
            assert r[0, 1] == pytest.approx(m_b, rel=1e-7)


def test_residual_lag_two_needs_three_steps(B):
    pb = problem(40, 30, "closed")
    dom = B.Domain(pb, "fp64")
    upload(dom, seeded_state(pb, 3))
    dom.set_residual_lag(2)
    dom.step(2)
    assert math.isinf(dom.residual()[0])
    dom.step(3)
    assert math.isfinite(dom.residual()[0])
    with pytest.raises(B.AxlbmError):
        dom.set_residual_lag(3)
    dom.close()


def test_residual_single_steps_and_first_call(B):
    pb = problem(40, 30, "closed")
    dom = B.Domain(pb, "fp64")
    upload(dom, seeded_state(pb, 3))
    dom.step(1)
    assert math.isinf(dom.residual()[0])  # no previous level yet
    dom.step(1)
    assert math.isfinite(dom.residual()[0])
    dom.close()


def test_mass_budget_identity_on_gpu(B):
    """M(t+1) = M(t) - B(t) with the GPU's own FP64 reductions."""
    pb = problem(130, 66, "free-top")
    dom = B.Domain(pb, "fp64")
    upload(dom, seeded_state(pb, 8))
    dom.step(2)
    _, m0, b0 = dom.residual()
    for _ in range(5):
        dom.step(1)
        _, m1, b1 = dom.residual()
        assert abs(m1 - (m0 - b0)) <= 1e-12 * m0
        m0, b0 = m1, b1
    dom.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_set_fields_and_rest_state_match_oracle_equilibria(B, precision):
    pb = problem(65, 33, "crystal")
    fields = I.random_fields(pb.nr, pb.nz, seed=77)
    want = oracle.equilibrium(pb, fields)
    dom = B.Domain(pb, precision)
    f, g, h = dom.get_populations()
    rest = oracle.rest_state(pb)
    tol = 1e-15 if precision == "fp64" else 1e-7
    assert rel_err(f, rest.f) <= tol and rel_err(h, rest.h) <= tol and np.max(np.abs(g)) == 0.0
    dom.set_fields(fields)
    f, g, h = dom.get_populations()
    assert rel_err(f, want.f) <= 4 * tol and rel_err(g, want.g) <= 4 * tol and rel_err(h, want.h) <= 4 * tol
    import torch
    dev = torch.tensor(fields, dtype=torch.float32, device="cuda")
    dom.set_fields(dev)
    f, _, _ = dom.get_populations()
    assert rel_err(f, want.f) <= 1e-6
    dom.close()


def test_nonfinite_is_reported(B):
    pb = problem(20, 20, "closed")
    st = seeded_state(pb, 2)
    st.f[3, 10, 10] = np.nan
    dom = B.Domain(pb, "fp32")
    upload(dom, st)
    dom.step(2)
    with pytest.raises(B.AxlbmError) as ei:
        dom.residual()
    assert ei.value.status == B.ENONFINITE
    dom.close()


def test_hagen_poiseuille_on_gpu_fp64(B):
    """Hagen-Poiseuille pipe 32 x 8, tau = 0.8, u_max = 0.01 (FP64): the GPU
    reaches the Eq. 57 residual 1e-10 and the oracle's profile."""
    pb = I.hagen_poiseuille(nr=32, nz=8, tau=0.8, umax=0.01)
    dom = B.Domain(pb, "fp64")
    dom.step(25000)
    res, mass, _ = dom.residual()
    assert res <= 1e-10
    assert abs(mass - 256.0) <= 1e-10 * 256.0
    uz = dom.moments(B.UZ)[0]
    nu = (pb.tau - 0.5) / 3
    ua = A.hagen_poiseuille(oracle.node_radii(pb), 32, pb.az0, nu)
    err = math.sqrt(np.sum((uz[4] - ua) ** 2) / np.sum(ua ** 2))
    assert err <= 3e-3
    st = oracle.rest_state(pb)
    oracle.step(st, 25000)
    assert rel_err(uz, oracle.moments(st)[2]) <= 1e-10
    dom.close()


@pytest.mark.parametrize("precision", ["fp32"])
def test_full_size_sampled_parity(B, precision):
    """The benchmark's grid (pipe 4096 x 8192, D2Q9) in the benchmark's launch
    shape: after 1, 2 and 3 steps, sampled nodes (axis, wall, periodic ends,
    corners and random interior) match the oracle run on a window around them."""
    pb = I.large_pipe()
    fields = I.random_fields(pb.nr, pb.nz, seed=5)
    dom = B.Domain(pb, precision)
    dom.set_fields(fields)
    f0, g0, h0 = dom.get_populations()
    rng = np.random.default_rng(12)
    picks = [(0, 0), (0, pb.nz - 1), (pb.nr - 1, 0), (pb.nr - 1, pb.nz - 1), (1, 1), (pb.nr - 2, 5),
             (0, 4000), (pb.nr - 1, 333), (2047, 0), (2048, pb.nz - 1)]
    picks += [(int(rng.integers(0, pb.nr)), int(rng.integers(0, pb.nz))) for _ in range(20)]
    done = 0
    for steps in (1, 1, 1):
        dom.step(steps)
        done += steps
        f1, _, _ = dom.get_populations()
        for (j, k) in picks:
            want, _, _ = window_oracle((f0, g0, h0), pb, j, k, done, 0)
            assert np.max(np.abs(f1[:, k, j] - want)) <= POP_TOL[precision] * 0.5, (j, k, done)
    dom.close()


def test_low_viscosity_bgk_versus_mrt(B):
    """Sec. IV B's comparison: rotating-lid cylinder A = 1.5, Re = 1290, 100 x 150,
    tau = 0.005 (nu = 1.67e-3, s_v = 1/(0.5 + 0.005)).  The MRT scheme with
    s_e = s_v stays finite and converges; the BGK outcome is recorded."""
    import json
    import os
    nr, re_ = 100, 1290.0
    nu = 0.005 / 3.0
    omega = re_ * nu / nr ** 2
    base = I.Problem(nr=nr, nz=150, tau=0.505, z_lo="wall", z_hi="wall", swirl=True, omega={"hi": omega})
    out = {}
    for coll in ("bgk", "mrt"):
        pb = dataclasses.replace(base, collision=coll)
        dom = B.Domain(pb, "fp32")
        finite = True
        res = float("nan")
        for _ in range(40):
            dom.step(5000)
            res, _, _ = dom.residual(allow_nonfinite=True)
            if not np.isfinite(res):
                finite = False
                break
        out[coll] = {"finite": finite, "residual": res, "steps": dom.time}
        if coll == "mrt":
            uz_axis = dom.moments(B.UZ)[0][:, 0]
            out[coll]["uz_axis_max_over_omega_r"] = float(np.max(uz_axis) / (omega * nr))
        dom.close()
    record("low_viscosity.json", "bgk_versus_mrt", out)
    assert out["mrt"]["finite"], out


@pytest.mark.parametrize("mix", ["crystal", "nee-axis-node", "annulus-mixed"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_parity_after_1000_steps(B, mix, precision):
    """1000 steps from the same seeded state (swirl and temperature, the
    paper's axis variants and walls, BGK and MRT): every population within
    1e-10 (FP64) or 1e-5 (FP32) of the oracle, relative to the field's scale,
    after 10, 100 and 1000 steps."""
    pb = problem(70, 45, mix, collision="mrt" if mix.startswith("nee") else "bgk")
    worst, _ = run_and_compare(B, pb, precision, [10, 90, 900])
    assert max(worst.values()) <= POP_TOL[precision], worst
