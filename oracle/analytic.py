"""Closed-form solutions used to pin the oracle (TEST INFRASTRUCTURE).

Each function states the flow it solves.  None of them uses the lattice
Boltzmann scheme: they are the target solutions of the macroscopic equations
(Eqs. 1-4 and 52) that the scheme must reproduce.
"""
from __future__ import annotations

import math

import numpy as np


def hagen_poiseuille(r, radius: float, a: float, mu: float):
    """Eq. 55: u_z = U0 (1 - r^2/R^2) with U0 = a R^2 / (4 mu)."""
    r = np.asarray(r, dtype=np.float64)
    u0 = a * radius * radius / (4.0 * mu)
    return u0 * (1.0 - (r / radius) ** 2)


def j0(z, terms: int = 120):
    """Bessel J0 of a complex argument from its power series
    J0(z) = sum_k (-z^2/4)^k / (k!)^2, summed until the terms stop mattering."""
    z = np.asarray(z, dtype=np.complex128)
    q = -(z * z) / 4.0
    term = np.ones_like(z)
    acc = np.ones_like(z)
    for k in range(1, terms):
        term = term * q / float(k * k)
        acc = acc + term
        if np.all(np.abs(term) <= 1e-18 * np.maximum(np.abs(acc), 1e-300)):
            break
    return acc


def womersley(r, t, radius: float, a0: float, rho0: float, omega: float, mu: float):
    """Eq. 56: u_z = Re{ a0/(i rho0 omega) [1 - J0(r phi / R)/J0(phi)] e^{i omega t} },
    phi = (-alpha + i alpha)/sqrt(2), alpha = R sqrt(rho0 omega / mu)."""
    r = np.asarray(r, dtype=np.float64)
    alpha = radius * math.sqrt(rho0 * omega / mu)
    phi = (-alpha + 1j * alpha) / math.sqrt(2.0)
    shape = 1.0 - j0(r * phi / radius) / j0(np.asarray(phi))
    val = a0 / (1j * rho0 * omega) * shape * np.exp(1j * omega * t)
    return np.real(val)


def annular_poiseuille(r, r1: float, r2: float, a: float, mu: float):
    """Axial flow between coaxial cylinders r1 < r < r2 driven by a uniform
    axial force a: mu (u'' + u'/r) = -a, u(r1) = u(r2) = 0, so
    u = a/(4 mu) [r2^2 - r^2 - (r2^2 - r1^2) ln(r2/r) / ln(r2/r1)]."""
    r = np.asarray(r, dtype=np.float64)
    c = a / (4.0 * mu)
    return c * (r2 * r2 - r * r - (r2 * r2 - r1 * r1) * np.log(r2 / r) / math.log(r2 / r1))


def taylor_couette(r, r1: float, r2: float, om1: float, om2: float):
    """Circular Couette flow: u_theta = A r + B / r with u_theta(r1) = om1 r1
    and u_theta(r2) = om2 r2 (steady solution of Eq. 52 with u_r = u_z = 0)."""
    r = np.asarray(r, dtype=np.float64)
    a = (om2 * r2 * r2 - om1 * r1 * r1) / (r2 * r2 - r1 * r1)
    b = (om1 - om2) * r1 * r1 * r2 * r2 / (r2 * r2 - r1 * r1)
    return a * r + b / r


def radial_conduction(r, r1: float, r2: float, t1: float, t2: float):
    """Steady conduction between coaxial cylinders: T = t1 + (t2 - t1) ln(r/r1)/ln(r2/r1)."""
    r = np.asarray(r, dtype=np.float64)
    return t1 + (t2 - t1) * np.log(r / r1) / math.log(r2 / r1)


def xi(u, ua) -> float:
    """Relative error of Sec. IV A: sum |u - u_a| / sum |u_a| over radial nodes."""
    u = np.asarray(u)
    ua = np.asarray(ua)
    return float(np.sum(np.abs(u - ua)) / np.sum(np.abs(ua)))
