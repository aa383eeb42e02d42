"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  Each one is chosen so that a plausible slip
in the oracle (a dropped term, a flipped sign, a wrong index, a transposed
operand) fails at least one of them:

* the per-node mass budget sum f* - sum f = -rho u_r / r (follows from
  Eqs. 12-17) catches mistakes in the density, the u_r/r source and the
  radius-dependent rate;
* the Cartesian limit r -> infinity must give the textbook BGK update with the
  He-Shan-Doolen force and its trapezoidal shift (Eqs. 8 and 13 without the
  1/r terms) and the plain D2Q4 advection-diffusion update (Eq. 53);
* streaming must be a one-to-one map of populations under every boundary mix,
  and individual moves are checked against hand-derived tables;
* closed-form flows: Hagen-Poiseuille (Eq. 55), Womersley (Eq. 56) at the
  paper's own parameters, annular Poiseuille, Taylor-Couette (Eq. 52) and
  radial conduction, with second-order convergence where the axis is absent;
* solid-body rotation tests the inertial force of Sec. III C.
"""
import math
import os

import numpy as np
import pytest

from oracle import analytic as A
from paper_1003_0282_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")

# Textbook D2Q9 / D2Q4 tables in the oracle's population order, (r, z) components.
E9 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
E4 = np.array([(1, 0), (0, 1), (-1, 0), (0, -1)], float)


def golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            out[key] = float(val)
    return out


def near_eq(rng, rho=1.0, u=(0.02, -0.03), noise=0.05):
    eu = E9 @ np.asarray(u)
    feq = W9 * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * float(np.dot(u, u)))
    return feq * (1 + noise * rng.uniform(-1, 1, 9))


# ----------------------------------------------------------------------------- paper numbers


def test_golden_paper_parameters_are_consistent():
    g = golden()
    # Eq. 55: U0 = a R^2 / (4 mu)
    assert g["hp_a"] * g["hp_R"] ** 2 / (4 * g["hp_mu"]) == pytest.approx(g["hp_U0"], rel=1e-12)
    # Womersley number and Reynolds number of Sec. IV A
    omega = 2 * math.pi / g["wom_T"]
    alpha = g["wom_R"] * math.sqrt(omega / g["wom_mu"])
    assert alpha == pytest.approx(g["wom_alpha"], abs=5e-4)
    uc = g["wom_a0"] * alpha ** 2 / (4 * omega)
    assert uc * 2 * g["wom_R"] / g["wom_mu"] == pytest.approx(g["wom_Re"], rel=1e-3)


def test_j0_series_matches_scipy():
    special = pytest.importorskip("scipy.special")
    for alpha in (0.5, 2.0, 5.0, 7.927, 10.0):
        phi = (-alpha + 1j * alpha) / math.sqrt(2)
        z = np.linspace(0, 1, 33) * phi
        ours = A.j0(z)
        ref = special.jv(0, z)
        assert np.max(np.abs(ours - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_womersley_small_alpha_is_quasi_steady_poiseuille():
    radius, mu, a0 = 20.0, 0.1, 1e-5
    omega = 1e-9  # alpha ~ 2e-3
    r = np.linspace(0, radius, 11)
    u = A.womersley(r, 0.0, radius, a0, 1.0, omega, mu)
    assert np.allclose(u, A.hagen_poiseuille(r, radius, a0, mu), rtol=1e-6, atol=1e-14)


# ----------------------------------------------------------------------------- one node


@pytest.mark.parametrize("swirl,temp", [(False, False), (True, False), (True, True)])
def test_collision_mass_budget_identity(orc, swirl, temp):
    """sum_a f*_a - sum_a f_a = -rho u_r / r for every node (Eqs. 12-17)."""
    rng = np.random.default_rng(7)
    pb = I.Problem(nr=4, nz=4, tau=0.8, swirl=swirl, temperature=temp, tau_t=0.7,
                   az0=3e-5, gbeta=1e-4, t_ref=0.5)
    for _ in range(50):
        r = float(rng.uniform(0.5, 40.0))
        f = near_eq(rng, rho=rng.uniform(0.95, 1.05), u=rng.uniform(-0.05, 0.05, 2))
        g = rng.uniform(-0.01, 0.01, 4)
        h = rng.uniform(0.1, 0.2, 4)
        fo, go, ho, mom = orc.collide_cell(pb, r, 3e-5, f, g, h)
        lhs = fo.sum() - f.sum()
        rhs = -mom[0] * mom[1] / r
        assert abs(lhs - rhs) <= 2e-15 * f.sum()


def test_collision_reduces_to_cartesian_bgk_far_from_axis(orc):
    """As r -> infinity every 1/r term vanishes: the update must equal the
    textbook BGK collision with the He-Shan-Doolen force and the trapezoidal
    shift (omega = 1/tau_s, u = (sum e f + F/2)/rho), and D2Q4 advection-
    diffusion for g (Eq. 53 with S^g -> 0)."""
    rng = np.random.default_rng(11)
    tau_s, a, rho0 = 0.83, 2e-5, 1.0
    pb = I.Problem(nr=4, nz=4, tau=tau_s, swirl=True, rho0=rho0, az0=a)
    for _ in range(20):
        f = near_eq(rng, rho=rng.uniform(0.97, 1.03), u=rng.uniform(-0.04, 0.04, 2))
        g = rng.uniform(-0.01, 0.01, 4)
        fo, go, _, _ = orc.collide_cell(pb, 1e12, a, f, g)
        # textbook, written independently of the oracle
        F = np.array([0.0, a])
        rho = f.sum()
        u = (E9.T @ f + 0.5 * F) / rho
        eu = E9 @ u
        feq = W9 * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u @ u)
        om = 1.0 / tau_s
        force = 3.0 * ((E9 - u) @ F) / rho * feq
        ref = f - om * (f - feq) + (1 - 0.5 * om) * force
        assert np.max(np.abs(fo - ref)) <= 1e-12
        uth = g.sum() / rho0
        geq = rho0 * uth / 4 * (1 + 2 * (E4 @ u))
        taug = 2 * (tau_s - 0.5) / 3
        gref = g - (g - geq) / (taug + 0.5)
        assert np.max(np.abs(go - gref)) <= 1e-12


def test_source_zeroth_moments_at_equilibrium(orc):
    """With g and h at their equilibria only the sources act, and their zeroth
    moments are the macroscopic source terms: sum S^g = -(2 u_r / r + nu / r^2)
    rho0 u_theta (Eq. 52 divided through, nu = tau_g / 2) and sum S^T =
    -(u_r / r) T (conservative advection-diffusion with div u = -u_r / r)."""
    rng = np.random.default_rng(5)
    rho0, tau_s = 1.3, 0.9
    pb = I.Problem(nr=4, nz=4, tau=tau_s, rho0=rho0, swirl=True, temperature=True, tau_t=0.7)
    nu = (2 * (tau_s - 0.5) / 3) / 2
    for _ in range(30):
        r = float(rng.uniform(0.5, 20.0))
        f = near_eq(rng, rho=rho0 * rng.uniform(0.97, 1.03), u=rng.uniform(-0.05, 0.05, 2))
        g0 = rng.uniform(-0.01, 0.01, 4)
        h0 = rng.uniform(0.1, 0.2, 4)
        uth, temp = float(rng.uniform(-0.02, 0.02)), float(rng.uniform(0.2, 0.8))
        g, h = g0, h0
        for _ in range(6):  # u_r depends on u_theta (half inertial force): iterate to a fixed point
            _, _, _, mom = orc.collide_cell(pb, r, 0.0, f, g, h)
            u = mom[1:3]
            g = rho0 * uth / 4 * (1 + 2 * (E4 @ u))   # textbook D2Q4 equilibria
            h = temp / 4 * (1 + 2 * (E4 @ u))
        _, go, ho, mom2 = orc.collide_cell(pb, r, 0.0, f, g, h)
        assert mom2[3] == pytest.approx(uth, rel=1e-13, abs=1e-17)
        assert mom2[4] == pytest.approx(temp, rel=1e-13)
        ur = mom2[1]
        assert go.sum() - g.sum() == pytest.approx(-(2 * ur / r + nu / r ** 2) * rho0 * uth,
                                                   rel=1e-10, abs=1e-18)
        assert ho.sum() - h.sum() == pytest.approx(-(ur / r) * temp, rel=1e-10, abs=1e-18)


def test_momentum_gain_far_from_axis_is_the_force(orc):
    """Far from the axis one step adds exactly F to sum e f (the trapezoidal
    scheme of Eqs. 8/13): F_z = a + rho0 g beta (T - T_ref) with buoyancy."""
    rng = np.random.default_rng(9)
    a, gbeta, t_ref, rho0 = 3e-6, 2e-4, 0.4, 1.1
    pb = I.Problem(nr=4, nz=4, tau=0.7, rho0=rho0, temperature=True, tau_t=0.8,
                   gbeta=gbeta, t_ref=t_ref, az0=a)
    for _ in range(20):
        f = near_eq(rng, rho=rho0, u=rng.uniform(-0.03, 0.03, 2))
        h = rng.uniform(0.05, 0.25, 4)
        fo, _, _, _ = orc.collide_cell(pb, 1e12, a, f, None, h)
        fz = a + rho0 * gbeta * (h.sum() - t_ref)
        assert (E9[:, 1] @ fo) - (E9[:, 1] @ f) == pytest.approx(fz, rel=1e-9)
        assert (E9[:, 0] @ fo) - (E9[:, 0] @ f) == pytest.approx(0.0, abs=1e-14)


def test_force_is_taken_at_the_pre_collision_time(orc):
    """The axial force of step n is a(n) = az0 cos(omega_t n), at the
    pre-collision time.  One step from rest at time t0 adds exactly a(t0) to
    sum e_z f of a node whose neighbours are fluid at rest too (far from the
    axis, where the 1/r terms vanish), and not a(t0 + 1)."""
    az0, om, t0 = 2e-5, 0.3, 5
    pb = I.Problem(nr=5, nz=4, tau=0.8, inner="wall", r0=1e12, z_lo="periodic", z_hi="periodic",
                   az0=az0, omega_t=om)
    st = orc.rest_state(pb)
    st.t = t0
    orc.step(st, 1)
    gain = E9[:, 1] @ st.f[:, :, 2]  # middle column, every row
    assert np.allclose(gain, az0 * np.cos(om * t0), rtol=1e-9, atol=0)
    assert not np.allclose(gain, az0 * np.cos(om * (t0 + 1)), rtol=1e-3, atol=0)


# ----------------------------------------------------------------------------- streaming

BOUNDARY_MIXES = [
    dict(inner="axis", z_lo="periodic", z_hi="periodic"),
    dict(inner="axis", z_lo="wall", z_hi="wall"),
    dict(inner="axis", z_lo="wall", z_hi="free"),
    dict(inner="axis", z_lo="wall", z_hi="mixed", r_split=2.7),
    dict(inner="wall", r0=3.0, z_lo="wall", z_hi="mixed", r_split=5.0),
    dict(inner="wall", r0=1.0, z_lo="periodic", z_hi="periodic"),
]


@pytest.mark.parametrize("mix", BOUNDARY_MIXES)
@pytest.mark.parametrize("shape", [(5, 4), (1, 3), (3, 1), (1, 1)])
def test_stream_is_one_to_one(orc, mix, shape):
    """Every post-collision population lands in exactly one slot."""
    nr, nz = shape
    pb = I.Problem(nr=nr, nz=nz, tau=0.8, swirl=True, temperature=True, **mix)
    n = nr * nz
    fp = (np.arange(9 * n, dtype=float) + 1.0).reshape(9, nz, nr)
    gp = (np.arange(4 * n, dtype=float) + 1.0).reshape(4, nz, nr)
    fn, gn, hn = orc.stream(pb, fp, gp, gp)
    assert not np.isnan(fn).any() and not np.isnan(gn).any() and not np.isnan(hn).any()
    assert np.array_equal(np.sort(fn.ravel()), np.sort(fp.ravel()))
    # with resting walls g is only permuted up to sign; h on adiabatic faces is permuted
    assert np.array_equal(np.sort(np.abs(gn.ravel())), np.sort(gp.ravel()))
    assert np.array_equal(np.sort(hn.ravel()), np.sort(gp.ravel()))


def _codes(nr, nz, q):
    # code(a, k, j) = 100 a + 10 k + j + 1
    a, k, j = np.meshgrid(np.arange(q), np.arange(nz), np.arange(nr), indexing="ij")
    return 100.0 * a + 10.0 * k + j + 1.0


def code(a, k, j):
    return 100.0 * a + 10.0 * k + j + 1.0


def test_stream_table_axis_wall_periodic(orc):
    pb = I.Problem(nr=3, nz=3, tau=0.8)
    fn, _, _ = orc.stream(pb, _codes(3, 3, 9))
    assert fn[1, 1, 1] == code(1, 1, 0)  # plain move
    assert fn[2, 0, 1] == code(2, 2, 1)  # periodic wrap in z
    assert fn[1, 1, 0] == code(3, 1, 0)  # specular reflection at the axis
    assert fn[5, 1, 0] == code(6, 0, 0)  # (-1,1) from (0,0) comes back as (1,1) at (0,1)
    assert fn[8, 1, 0] == code(7, 2, 0)  # (-1,-1) from (0,2) comes back as (1,-1) at (0,1)
    assert fn[3, 1, 2] == code(1, 1, 2)  # bounce-back at the outer wall
    assert fn[6, 1, 2] == code(8, 1, 2)
    assert fn[7, 1, 2] == code(5, 1, 2)


def test_stream_table_lids_free_surface_corners(orc):
    pb = I.Problem(nr=3, nz=3, tau=0.8, z_lo="wall", z_hi="free")
    fn, _, _ = orc.stream(pb, _codes(3, 3, 9))
    assert fn[2, 0, 1] == code(4, 0, 1)  # bottom wall bounce-back
    assert fn[5, 0, 1] == code(7, 0, 1)
    assert fn[6, 0, 1] == code(8, 0, 1)
    assert fn[4, 2, 1] == code(2, 2, 1)  # free surface: mirror in z
    assert fn[8, 2, 1] == code(5, 2, 0)
    assert fn[7, 2, 1] == code(6, 2, 2)
    assert fn[8, 2, 0] == code(6, 2, 0)  # axis + free surface corner: double mirror
    assert fn[5, 0, 0] == code(7, 0, 0)  # axis + wall corner: bounce-back
    assert fn[7, 2, 2] == code(5, 2, 2)  # outer wall + free surface corner: bounce-back


def test_stream_table_mixed_top(orc):
    # crystal disk r < 1.0: crossing radii 0.5 (column 0 vertical) and 0.0 are wall,
    # 1.0 (between columns 0 and 1) and beyond are free surface
    pb = I.Problem(nr=3, nz=3, tau=0.8, z_lo="wall", z_hi="mixed", r_split=1.0)
    fn, _, _ = orc.stream(pb, _codes(3, 3, 9))
    assert fn[4, 2, 0] == code(2, 2, 0)  # vertical under the disk: bounce-back
    assert fn[4, 2, 1] == code(2, 2, 1)  # vertical under the free surface: mirror (same slot)
    assert fn[8, 2, 1] == code(5, 2, 0)  # crossing at r = 1: free, mirror in z
    assert fn[7, 2, 0] == code(6, 2, 1)
    assert fn[8, 2, 0] == code(6, 2, 0)  # crossing at r = 0 (axis corner): wall


def test_stream_table_swirl_and_temperature_walls(orc):
    om_out, om_lo, tw = 0.003, 0.002, 0.7
    pb = I.Problem(nr=3, nz=3, tau=0.8, z_lo="wall", z_hi="free", swirl=True, temperature=True,
                   rho0=1.2, omega={"outer": om_out, "lo": om_lo}, t_wall={"outer": tw})
    gp = _codes(3, 3, 4)
    fn, gn, hn = orc.stream(pb, _codes(3, 3, 9), gp, gp)
    # D2Q4 order: (1,0), (0,1), (-1,0), (0,-1)
    assert gn[2, 1, 2] == pytest.approx(-code(0, 1, 2) + 0.5 * 1.2 * om_out * 3.0)  # moving side wall
    assert gn[0, 1, 0] == -code(2, 1, 0)  # axis: u_theta is odd in r
    assert gn[1, 0, 1] == pytest.approx(-code(3, 0, 1) + 0.5 * 1.2 * om_lo * 1.5)  # moving lid at r = 1.5
    assert gn[3, 2, 1] == code(1, 2, 1)  # free surface: zero normal gradient
    assert hn[2, 1, 2] == pytest.approx(-code(0, 1, 2) + 0.5 * tw)  # Dirichlet wall
    assert hn[1, 0, 1] == code(3, 0, 1)  # adiabatic lid
    assert hn[0, 1, 0] == code(2, 1, 0)  # axis: symmetric


# ----------------------------------------------------------------------------- whole domains


@pytest.mark.parametrize("mix", BOUNDARY_MIXES)
def test_global_mass_budget(orc, mix):
    """Streaming under bounce-back, mirror and periodic rules conserves sum f, so
    M(t+1) = M(t) - sum_cells rho u_r / r exactly (to rounding)."""
    nr, nz = 12, 10
    pb = I.Problem(nr=nr, nz=nz, tau=0.75, swirl=True, temperature=True, tau_t=0.7,
                   az0=1e-5, omega_t=0.01, gbeta=1e-4, t_ref=0.5,
                   omega={"outer": 0.002, "lo": -0.001, "hi": 0.003}, t_wall={"outer": 1.0},
                   **mix)
    fields = I.random_fields(nr, nz, seed=3)
    st = orc.equilibrium(pb, fields)
    st.f *= I.random_noise(st.f.shape, seed=4, amplitude=0.01)
    for _ in range(30):
        m0, b0, _ = orc.stats(st)
        orc.step(st, 1)
        m1, _, _ = orc.stats(st)
        assert abs(m1 - (m0 - b0)) <= 1e-13 * m0


def _hp_error(orc, nr, tau=0.8, umax=0.01):
    pb = I.hagen_poiseuille(nr=nr, nz=1, tau=tau, umax=umax)
    st = orc.rest_state(pb)
    nu = (tau - 0.5) / 3
    orc.step(st, int(16 * nr * nr / (nu * 5.783)))
    m = orc.moments(st)
    ua = A.hagen_poiseuille(orc.node_radii(pb), nr, pb.az0, pb.rho0 * nu)
    return math.sqrt(np.sum((m[2, 0] - ua) ** 2) / np.sum(ua ** 2)), st, m


def test_hagen_poiseuille_closed_form(orc):
    err, st, m = _hp_error(orc, 32)
    assert err <= 3e-3
    assert np.max(np.abs(m[1])) <= 1e-13  # u_r stays zero
    mass0, _, _ = orc.stats(st)
    assert abs(mass0 - 32.0) <= 1e-11 * 32.0  # u_r = 0 up to rounding over ~28k steps
    orc.step(st, 1000)
    mass1, _, speed0 = orc.stats(st)
    assert abs(mass1 - mass0) <= 1e-12 * mass0  # mass conserved to 1e-12 relative
    orc.step(st, 1)
    _, _, speed1 = orc.stats(st)
    assert np.max(np.abs(speed1 - speed0)) <= 1e-10  # Eq. 57 residual at steady state


def test_hagen_poiseuille_paper_case(orc):
    """The paper's own Hagen-Poiseuille parameters (Sec. IV A): R = 20, a = 1e-4,
    mu = 0.2 (so tau_s = 1.1), U0 = 0.05, here on the half-spacing grid with a
    bounce-back wall: the profile must match Eq. 55 within 2 % of U0.  (With
    tau_s > 1 the inward rate of Eq. 13 at r = 1/2 drops below zero; the
    update stays stable for this flow.)"""
    g = golden()
    radius = int(g["hp_R"])
    tau_s = 3 * g["hp_mu"] + 0.5
    pb = I.Problem(nr=radius, nz=1, tau=tau_s, az0=g["hp_a"])
    st = orc.rest_state(pb)
    orc.step(st, 30000)
    m = orc.moments(st)
    ua = A.hagen_poiseuille(orc.node_radii(pb), radius, g["hp_a"], g["hp_mu"])
    assert ua[0] == pytest.approx(g["hp_U0"] * (1 - 0.25 / radius ** 2))
    assert np.max(np.abs(m[2, 0] - ua)) <= 0.02 * g["hp_U0"]


def test_hagen_poiseuille_convergence(orc):
    """Half-spacing specular axis: the error falls at an observed order that
    climbs towards 2 (about 1.5-1.7 on these grids; see the annulus tests for
    the bulk scheme's clean order 2)."""
    errs = [_hp_error(orc, n)[0] for n in (8, 16, 32)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(o >= 1.4 for o in orders)
    assert orders[1] >= orders[0]


def _order(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_annular_poiseuille_second_order(orc):
    errs = []
    for nr in (8, 16, 32):
        r1, nu = 0.5 * nr, 0.1
        a = 1e-3 / nr ** 2
        pb = I.Problem(nr=nr, nz=1, tau=3 * nu + 0.5, r0=r1, inner="wall", az0=a)
        st = orc.rest_state(pb)
        orc.step(st, int(16 * nr * nr / (nu * 5.783)))
        ua = A.annular_poiseuille(orc.node_radii(pb), r1, r1 + nr, a, nu)
        errs.append(np.sqrt(np.mean((orc.moments(st)[2, 0] - ua) ** 2)) / ua.max())
    assert all(abs(o - 2.0) <= 0.1 for o in _order(errs))


def test_taylor_couette_second_order(orc):
    errs = []
    for nr in (8, 16, 32):
        r1, nu = 0.5 * nr, 0.1
        om1, om2 = 0.01 / r1, -0.004 / (r1 + nr)
        pb = I.Problem(nr=nr, nz=1, tau=3 * nu + 0.5, r0=r1, inner="wall", swirl=True,
                       omega={"inner": om1, "outer": om2})
        st = orc.rest_state(pb)
        orc.step(st, int(16 * nr * nr / (nu * 5.783)))
        ua = A.taylor_couette(orc.node_radii(pb), r1, r1 + nr, om1, om2)
        errs.append(np.sqrt(np.mean((orc.moments(st)[3, 0] - ua) ** 2)) / 0.01)
    assert all(abs(o - 2.0) <= 0.1 for o in _order(errs))


def test_radial_conduction_second_order(orc):
    errs = []
    for nr in (8, 16, 32):
        r1, tau_t = 0.5 * nr, 0.8
        kappa = (tau_t - 0.5) / 2
        pb = I.Problem(nr=nr, nz=1, tau=0.8, r0=r1, inner="wall", temperature=True, tau_t=tau_t,
                       t_wall={"inner": 1.0, "outer": 0.0})
        st = orc.rest_state(pb, t_init=0.5)
        orc.step(st, int(16 * nr * nr / (kappa * 5.783)))
        ua = A.radial_conduction(orc.node_radii(pb), r1, r1 + nr, 1.0, 0.0)
        errs.append(np.sqrt(np.mean((orc.moments(st)[4, 0] - ua) ** 2)))
    assert all(abs(o - 2.0) <= 0.1 for o in _order(errs))


def test_womersley_paper_case(orc):
    """Sec. IV A: R = 20, T = 1200, mu = 0.1/3, a0 = 1e-3/3, alpha = 7.927,
    ten periods from rest; <xi> over the tenth period.  The paper reports
    0.33 % with a node on the axis and Zou-He walls; half-spacing with
    bounce-back must stay within 1 %."""
    g = golden()
    radius, period, mu = int(g["wom_R"]), int(g["wom_T"]), g["wom_mu"]
    pb = I.Problem(nr=radius, nz=1, tau=3 * mu + 0.5, az0=g["wom_a0"], omega_t=2 * math.pi / period)
    st = orc.rest_state(pb)
    orc.step(st, (int(g["wom_periods"]) - 1) * period)
    r = orc.node_radii(pb)
    xis = []
    for n in range(16):
        orc.step(st, (int(g["wom_periods"]) - 1) * period + n * period // 16 - st.t)
        ua = A.womersley(r, st.t, radius, pb.az0, 1.0, pb.omega_t, mu)
        xis.append(A.xi(orc.moments(st)[2, 0], ua))
    assert np.mean(xis) <= 0.01


def test_solid_body_rotation_and_inertial_force(orc):
    """A closed cylinder whose walls all turn at Omega spins up to u_theta = Omega r;
    the inertial force rho0 u_theta^2 / r (Sec. III C) must then be balanced by
    the pressure gradient c_s^2 d rho / dr = rho0 Omega^2 r."""
    nr, nz, nu = 16, 16, 0.1
    om = 0.02 / nr
    pb = I.Problem(nr=nr, nz=nz, tau=3 * nu + 0.5, z_lo="wall", z_hi="wall", swirl=True,
                   omega={"outer": om, "lo": om, "hi": om})
    st = orc.rest_state(pb)
    orc.step(st, 12000)
    m = orc.moments(st)
    r = orc.node_radii(pb)
    mid = nz // 2
    err = np.abs(m[3, mid] - om * r) / (om * nr)
    assert np.max(err) <= 1e-2       # the two nodes next to the axis carry ~0.8 %
    assert np.max(err[3:]) <= 1e-3   # away from the axis
    assert np.max(np.abs(m[1:3])) <= 1e-4 * om * nr  # no meridional flow beyond O(Ma^2)
    drho = np.diff(m[0, mid]) / 3.0
    rmid = 0.5 * (r[1:] + r[:-1])
    expect = pb.rho0 * om * om * rmid
    assert np.max(np.abs(drho - expect)) <= 0.05 * np.max(expect)


def test_oracle_rejects_inconsistent_problems(orc):
    assert orc.validate(I.Problem(nr=4, nz=4, tau=0.8))
    assert not orc.validate(I.Problem(nr=4, nz=4, tau=0.4))
    assert not orc.validate(I.Problem(nr=4, nz=4, tau=0.8, r0=2.0, inner="axis"))
    assert not orc.validate(I.Problem(nr=4, nz=4, tau=0.8, z_lo="periodic", z_hi="wall"))
    assert not orc.validate(I.Problem(nr=0, nz=4, tau=0.8))


def test_equilibrium_reproduces_its_fields(orc):
    """Eqs. 6 and 54: sum f^eq = rho, sum e f^eq = rho u, sum g^eq = rho0 u_theta,
    sum h^eq = T.  Far from the axis and without forces the moments of Eqs.
    16-17 must therefore return the fields the equilibrium was built from."""
    pb = I.Problem(nr=9, nz=7, tau=0.8, r0=1e12, inner="wall", swirl=True, temperature=True, rho0=1.2)
    fields = I.random_fields(9, 7, seed=4, rho0=1.2)
    st = orc.equilibrium(pb, fields)
    got = orc.moments(st)
    for q in range(5):
        assert np.max(np.abs(got[q] - fields[q])) <= 1e-12 * max(1.0, np.max(np.abs(fields[q]))), q


def test_residual_speed_is_the_meridional_speed(orc):
    """Eq. 57 measures |u_p| = sqrt(u_z^2 + u_r^2): the azimuthal velocity is
    not part of it.  Far from the axis (where the 1/r terms of Eqs. 15-16 are
    negligible) an equilibrium built from fields (u_r, u_z, u_theta) must give
    the speed hypot(u_r, u_z) -- and 0 when only u_theta is non-zero, where a
    speed that included u_theta would be |u_theta|."""
    pb = I.Problem(nr=6, nz=5, tau=0.8, r0=1e6, inner="wall", swirl=True)
    fields = np.zeros((5, 5, 6))
    fields[0] = 1.0
    fields[4] = pb.t_ref
    rng = np.random.default_rng(57)
    fields[1] = rng.uniform(-0.03, 0.03, (5, 6))
    fields[2] = rng.uniform(-0.03, 0.03, (5, 6))
    fields[3] = rng.uniform(0.02, 0.05, (5, 6))
    _, _, speed = orc.stats(orc.equilibrium(pb, fields))
    assert np.max(np.abs(speed - np.hypot(fields[1], fields[2]))) <= 1e-8
    fields[1] = fields[2] = 0.0
    _, _, speed = orc.stats(orc.equilibrium(pb, fields))
    assert np.max(speed) <= 1e-8
