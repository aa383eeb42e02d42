"""Pins of the oracle's MRT collision (Sec. III B, Eqs. 37-51).

* the moment basis is orthogonal and maps the equilibrium of Eq. 6 to the
  m^eq of Eq. 39 (the paper does not print M; this pins the reading);
* far from the axis the update is the textbook semi-implicit MRT update with
  the moment-space force of Eq. 51, written here independently;
* with every rate equal it is the BGK update of the same force (up to the
  O(u^2 F) terms by which the two force terms differ);
* the per-node mass budget of Eqs. 12-17 holds unchanged;
* Hagen-Poiseuille converges at second order (the momentum correction of
  Eqs. 49-50 recovers the mu/r terms), and the paper's Womersley case reaches
  <xi> close to its 0.33 %.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import analytic as A
from paper_1003_0282_gb300 import inputs as I

E9 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def textbook_basis():
    ex, ey = E9[:, 0], E9[:, 1]
    e2 = ex ** 2 + ey ** 2
    return np.array([np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, ex, (-5 + 3 * e2) * ex, ey,
                     (-5 + 3 * e2) * ey, ex ** 2 - ey ** 2, ex * ey])


def feq(rho, u):
    eu = E9 @ u
    return W9 * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u @ u)


def test_moment_basis_is_orthogonal_and_gives_eq39(orc):
    M = orc.mrt_matrix()
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)), atol=1e-13)
    rng = np.random.default_rng(2)
    for _ in range(10):
        rho, u = rng.uniform(0.9, 1.1), rng.uniform(-0.05, 0.05, 2)
        want = rho * np.array([1, -2 + 3 * u @ u, 1 - 3 * u @ u, u[0], -u[0], u[1], -u[1], u[0] ** 2 - u[1] ** 2,
                               u[0] * u[1]])
        assert np.allclose(M @ feq(rho, u), want, atol=1e-14)


def test_mrt_far_from_axis_is_textbook_mrt(orc):
    rng = np.random.default_rng(3)
    tau_s, a, s_eps, s_q = 0.9, 1e-5, 1.3, 1.7
    pb = I.Problem(nr=4, nz=4, tau=tau_s, az0=a, collision="mrt", s_eps=s_eps, s_q=s_q)
    M = textbook_basis()
    sv = 1 / tau_s
    L = np.array([1, sv, s_eps, 1, s_q, 1, s_q, sv, sv])
    for _ in range(20):
        f = feq(rng.uniform(0.97, 1.03), rng.uniform(-0.04, 0.04, 2)) * (1 + 0.03 * rng.uniform(-1, 1, 9))
        fo, _, _, _ = orc.collide_cell(pb, 1e12, a, f)
        F = np.array([0.0, a])
        rho = f.sum()
        u = (E9.T @ f + 0.5 * F) / rho
        m = M @ f
        meq = M @ feq(rho, u)
        uF = u @ F
        S = np.array([0, 6 * uF, -6 * uF, F[0], -F[0], F[1], -F[1], 2 * (u[0] * F[0] - u[1] * F[1]),
                      u[0] * F[1] + u[1] * F[0]])
        mp = m - L * (m - meq) + (1 - 0.5 * L) * S
        ref = np.linalg.solve(M, mp)
        assert np.max(np.abs(fo - ref)) <= 1e-12


def test_mrt_with_equal_rates_is_bgk_far_from_axis(orc):
    rng = np.random.default_rng(4)
    tau_s, a = 0.75, 2e-6
    bgk = I.Problem(nr=4, nz=4, tau=tau_s, az0=a)
    mrt = dataclasses.replace(bgk, collision="mrt", s_eps=1 / tau_s, s_q=1 / tau_s)
    for _ in range(10):
        f = feq(1.0, rng.uniform(-0.02, 0.02, 2)) * (1 + 0.02 * rng.uniform(-1, 1, 9))
        fb, _, _, mom = orc.collide_cell(bgk, 1e12, a, f)
        fm, _, _, _ = orc.collide_cell(mrt, 1e12, a, f)
        # the two force terms agree up to O(u^2 F)
        bound = 3.0 * (mom[1] ** 2 + mom[2] ** 2) * a + 1e-15
        assert np.max(np.abs(fb - fm)) <= bound


def test_mrt_mass_budget_identity(orc):
    rng = np.random.default_rng(5)
    pb = I.Problem(nr=4, nz=4, tau=0.7, swirl=True, collision="mrt", az0=1e-5, s_eps=1.1, s_q=1.6)
    for _ in range(30):
        r = float(rng.uniform(0.5, 30))
        f = feq(rng.uniform(0.95, 1.05), rng.uniform(-0.05, 0.05, 2)) * (1 + 0.05 * rng.uniform(-1, 1, 9))
        fo, _, _, mom = orc.collide_cell(pb, r, 1e-5, f, rng.uniform(-0.01, 0.01, 4))
        assert abs(fo.sum() - f.sum() + mom[0] * mom[1] / r) <= 2e-15 * f.sum()


def _hp_mrt(orc, nr):
    pb = dataclasses.replace(I.hagen_poiseuille(nr=nr, nz=1, tau=0.8, umax=0.01), collision="mrt")
    st = orc.rest_state(pb)
    nu = (pb.tau - 0.5) / 3
    orc.step(st, int(16 * nr * nr / (nu * 5.783)))
    ua = A.hagen_poiseuille(orc.node_radii(pb), nr, pb.az0, nu)
    return math.sqrt(np.sum((orc.moments(st)[2, 0] - ua) ** 2) / np.sum(ua ** 2))


def test_mrt_hagen_poiseuille_second_order(orc):
    errs = [_hp_mrt(orc, n) for n in (8, 16, 32)]
    assert errs[-1] <= 1e-3
    assert all(abs(math.log2(errs[i] / errs[i + 1]) - 2.0) <= 0.1 for i in range(2))


def test_mrt_womersley_paper_case(orc):
    radius, period, mu = 20, 1200, 0.1 / 3
    pb = I.Problem(nr=radius, nz=1, tau=3 * mu + 0.5, az0=1e-3 / 3, omega_t=2 * math.pi / period, collision="mrt")
    st = orc.rest_state(pb)
    orc.step(st, 9 * period)
    r = orc.node_radii(pb)
    xis = []
    for n in range(16):
        orc.step(st, 9 * period + n * period // 16 - st.t)
        xis.append(A.xi(orc.moments(st)[2, 0], A.womersley(r, st.t, radius, pb.az0, 1.0, pb.omega_t, mu)))
    assert np.mean(xis) <= 0.005  # paper: 0.33 %


def test_mrt_equilibrium_state_is_rate_independent(orc):
    """A state with no non-equilibrium part, f = M^-1 (m^eq - S/2) (so that the
    unshifted f of Eq. 37 is at equilibrium), has m^(1) = 0: the correction of
    Eqs. 49-50 vanishes and Eq. 41 gives M^-1 (m^eq + S/2) for every choice of
    rates, at any radius."""
    M = textbook_basis()
    rng = np.random.default_rng(6)
    for _ in range(10):
        tau_s = float(rng.uniform(0.55, 1.2))
        rho, ur, uz, r = float(rng.uniform(0.95, 1.05)), float(rng.uniform(-0.03, 0.03)), \
            float(rng.uniform(-0.03, 0.03)), float(rng.uniform(0.5, 10.0))
        mu0 = (tau_s - 0.5) / 3.0
        fr, fz = -2.0 * mu0 * ur / r ** 2, 0.0
        meq = rho * np.array([1, -2 + 3 * (ur ** 2 + uz ** 2), 1 - 3 * (ur ** 2 + uz ** 2), ur, -ur, uz, -uz,
                              ur ** 2 - uz ** 2, ur * uz])
        uF = ur * fr + uz * fz
        S = -(ur / r) * meq + np.array([0, 6 * uF, -6 * uF, fr, -fr, fz, -fz, 2 * (ur * fr - uz * fz),
                                        ur * fz + uz * fr])
        f = np.linalg.solve(M, meq - 0.5 * S)
        want = np.linalg.solve(M, meq + 0.5 * S)
        for s_eps, s_q in ((1.1, 1.3), (1.6, 0.7), (0.0, 0.0)):
            pb = I.Problem(nr=4, nz=4, tau=tau_s, collision="mrt", s_eps=s_eps, s_q=s_q)
            fo, _, _, mom = orc.collide_cell(pb, r, 0.0, f)
            assert mom[1] == pytest.approx(ur, rel=1e-12, abs=1e-16) and mom[2] == pytest.approx(uz, rel=1e-12, abs=1e-16)
            assert np.max(np.abs(fo - want)) <= 1e-14


def test_mrt_momentum_correction_recovers_the_axisymmetric_viscous_terms(orc):
    """Chapman-Enskog check of Eqs. 45-50: give a node the first-order
    non-equilibrium moments of a chosen velocity gradient (Eq. 45), with rho
    and j consistent with Eqs. 14-15.  One collision must then change the
    momentum by the source plus exactly the terms the correction exists for:
    dj_r = S_3 + mu (2 du_r/dr) / r  (Eq. 47),  dj_z = S_5 + mu (du_z/dr + du_r/dz) / r
    (Eq. 48), mu = (1/s_v - 1/2) rho / 3."""
    M = textbook_basis()
    rng = np.random.default_rng(7)
    for _ in range(20):
        tau_s = float(rng.uniform(0.55, 1.2))
        sv = 1.0 / tau_s
        rho, ur, uz = float(rng.uniform(0.97, 1.03)), float(rng.uniform(-0.02, 0.02)), float(rng.uniform(-0.02, 0.02))
        r = float(rng.uniform(0.5, 8.0))
        a, b, c, d = rng.uniform(-1e-3, 1e-3, 4)  # du_r/dr, du_z/dz, du_z/dr, du_r/dz
        mu0 = (tau_s - 0.5) / 3.0
        fr, fz = -2.0 * mu0 * ur / r ** 2, 0.0
        u2 = ur ** 2 + uz ** 2
        meq = rho * np.array([1, -2 + 3 * u2, 1 - 3 * u2, ur, -ur, uz, -uz, ur ** 2 - uz ** 2, ur * uz])
        uF = ur * fr + uz * fz
        S = -(ur / r) * meq + np.array([0, 6 * uF, -6 * uF, fr, -fr, fz, -fz, 2 * (ur * fr - uz * fz),
                                        ur * fz + uz * fr])
        m1 = np.zeros(9)
        m1[1] = -2 * rho * (a + b) / sv                 # Eq. 45 with s_e = s_v
        m1[7] = -(2 * rho / 3) * (a - b) / sv
        m1[8] = -(rho / 3) * (c + d) / sv
        m1[2], m1[4], m1[6] = rng.uniform(-1e-4, 1e-4, 3)  # other non-hydrodynamic parts: arbitrary
        mbar = meq + m1 - 0.5 * S
        f = np.linalg.solve(M, mbar)
        pb = I.Problem(nr=4, nz=4, tau=tau_s, collision="mrt", s_eps=1.2, s_q=1.5)
        fo, _, _, mom = orc.collide_cell(pb, r, 0.0, f)
        assert mom[1] == pytest.approx(ur, rel=1e-12, abs=1e-16)
        mu = (1 / sv - 0.5) * rho / 3
        djr = E9[:, 0] @ (fo - f)
        djz = E9[:, 1] @ (fo - f)
        assert djr == pytest.approx(S[3] + mu * 2 * a / r, rel=1e-9, abs=1e-17)
        assert djz == pytest.approx(S[5] + mu * (c + d) / r, rel=1e-9, abs=1e-17)
