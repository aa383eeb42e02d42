"""Problem descriptions and seeded synthetic inputs.

This module is the only code that both the CUDA path and the FP64 oracle
consume.  It holds parameters and random numbers, none of the lattice
Boltzmann arithmetic: no equilibria, no moments, no collision, no streaming.

A :class:`Problem` describes one axisymmetric domain on the (r, z) half-plane:
``nr`` radial by ``nz`` axial nodes, node (j, k) at r = r0 + j + 1/2,
z = k + 1/2 (r = j with ``inner="axis_node"``).  Times are in lattice units
(dx = dt = 1).

``tau`` is the standard BGK relaxation time tau_s; the paper's tau (with
mu = tau rho c_s^2, Eq. 8 and the line after Eq. 36) is tau_s - 1/2.

Workload recipes follow the paper's test cases (Sec. IV): the Hagen-Poiseuille
pipe (Eq. 55), the Womersley pipe (Eq. 56), the lid-driven rotating cylinder
and Wheeler-type crystal-growth cells (Sec. IV B), plus the large pipe and the
uneven batch used for throughput measurements.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# inner face kinds
AXIS = "axis"            # axis halfway between node 0 and its mirror: r_j = j + 1/2
AXIS_NODE = "axis_node"  # node 0 on the axis: r_j = j (Sec. IV A)
WALL = "wall"
# axial face kinds (WALL too)
PERIODIC = "periodic"
FREE = "free"
MIXED = "mixed"  # top only: wall for r < r_split, free surface beyond
ZOU_HE = "zou_he"  # outer face only: Zou-He wall through the last column (pipes)
HALO = "halo"    # a cut through a larger domain (z-slab decomposition): populations cross to the neighbour slab
NEE = "nee"      # wet wall: the node row (or, as ``outer``, the last column) lies on the wall and is
                 # rebuilt by non-equilibrium extrapolation from its inner neighbour

FACES = ("inner", "outer", "lo", "hi")


@dataclasses.dataclass
class Problem:
    nr: int
    nz: int
    tau: float                      # standard relaxation time tau_s
    rho0: float = 1.0
    r0: float = 0.0                 # radius of the inner face (0: the axis)
    inner: str = AXIS
    z_lo: str = PERIODIC
    z_hi: str = PERIODIC
    outer: str = WALL               # WALL (half-way bounce-back), NEE (wet wall on column nr - 1) or
                                    # ZOU_HE (Zou-He wall through column nr - 1)
    swirl: bool = False
    temperature: bool = False
    tau_t: float = 0.8              # standard relaxation time of the temperature field
    az0: float = 0.0                # axial body force a(t) = az0 cos(omega_t t)
    omega_t: float = 0.0
    gbeta: float = 0.0              # Boussinesq coefficient g*beta
    t_ref: float = 0.0
    r_split: float = 0.0            # MIXED top: wall for r < r_split
    omega: Dict[str, float] = dataclasses.field(default_factory=dict)     # wall angular velocity per face
    t_wall: Dict[str, float] = dataclasses.field(default_factory=dict)    # Dirichlet temperature per face
    collision: str = "bgk"          # "bgk" (Eq. 13) or "mrt" (Eqs. 37-51)
    s_eps: float = 0.0              # MRT rate of epsilon (0: the default)
    s_q: float = 0.0                # MRT rate of q (0: the default)
    name: str = ""

    def omega_of(self, face: str) -> float:
        return float(self.omega.get(face, 0.0))

    def t_dirichlet(self, face: str) -> bool:
        return face in self.t_wall

    def t_value(self, face: str) -> float:
        return float(self.t_wall.get(face, 0.0))

    @property
    def cells(self) -> int:
        return self.nr * self.nz

    def node_radius(self, j):
        """Radius of column j (array or int)."""
        return self.r0 + np.asarray(j, dtype=np.float64) + (0.0 if self.inner == AXIS_NODE else 0.5)

    @property
    def wall_radius(self) -> float:
        """Radius of the outer wall (half-way, or on the last column for NEE)."""
        return float(self.node_radius(self.nr - 1)) + (0.0 if self.outer in (NEE, ZOU_HE) else 0.5)


# ----------------------------------------------------------------------------- recipes


def hagen_poiseuille(nr: int = 32, nz: int = 8, tau: float = 0.8, umax: float = 0.01,
                     rho0: float = 1.0) -> Problem:
    """Pipe of radius R = nr, periodic in z, bounce-back wall, constant axial
    force a chosen so that the Eq. 55 centre-line speed a R^2 / (4 mu) is umax."""
    nu = (tau - 0.5) / 3.0
    a = 4.0 * rho0 * nu * umax / float(nr) ** 2
    return Problem(nr=nr, nz=nz, tau=tau, rho0=rho0, az0=a, name=f"hagen-poiseuille {nr}x{nz}")


def womersley(nr: int = 64, nz: int = 4, tau: float = 0.8, alpha: float = 5.0,
              umax: float = 0.01, rho0: float = 1.0, period: Optional[int] = None) -> Problem:
    """Pipe driven by a = a0 cos(omega t) (Sec. IV A).  The period follows from
    alpha = R sqrt(omega / nu) unless given; a0 is set so that the amplitude of
    the quasi-steady centre-line speed a0 R^2/(4 mu) equals umax."""
    nu = (tau - 0.5) / 3.0
    if period is None:
        period = int(round(2.0 * math.pi * nr * nr / (alpha * alpha * nu)))
    omega = 2.0 * math.pi / period
    a0 = 4.0 * rho0 * nu * umax / float(nr) ** 2
    p = Problem(nr=nr, nz=nz, tau=tau, rho0=rho0, az0=a0, omega_t=omega,
                name=f"womersley {nr}x{nz} T={period}")
    p.period = period  # type: ignore[attr-defined]
    return p


def rotating_lid_cavity(nr: int = 128, aspect: float = 1.5, re: float = 990.0,
                        u_lid: float = 0.1, rho0: float = 1.0, collision: str = "bgk") -> Problem:
    """Closed cylinder of radius R = nr and height H = aspect R; the top lid
    rotates with Omega = u_lid / R, the bottom and side walls are at rest.
    Re = Omega R^2 / nu (Sec. IV B)."""
    nz = int(round(aspect * nr))
    omega = u_lid / nr
    nu = omega * nr * nr / re
    tau = 3.0 * nu + 0.5
    return Problem(nr=nr, nz=nz, tau=tau, rho0=rho0, z_lo=WALL, z_hi=WALL, swirl=True,
                   omega={"hi": omega}, collision=collision, name=f"cavity A={aspect} Re={re:g} {nr}x{nz}")


def wheeler_cell(nr: int = 128, re_x: float = 100.0, beta: float = 0.4, u_ref: float = 0.1,
                 re_c_ratio: float = -0.25, prandtl: float = 0.05, grashof: float = 1e4,
                 rho0: float = 1.0, collision: str = "bgk") -> Problem:
    """Wheeler-type Czochralski cell (Sec. IV B): crucible of radius R_c = nr and
    height H = R_c rotating with Omega_c (side wall and bottom), crystal disk
    of radius beta R_c on top rotating with Omega_x, free surface beyond it.
    Re_x = R_c^2 Omega_x / nu, crystal edge speed U_t = beta R_c Omega_x.  The
    thermal part (hot side wall T = 1, cold crystal T = 0, adiabatic elsewhere,
    Boussinesq force with Gr = g beta dT R^3 / nu^2, Pr = nu / kappa) is not in
    the paper.

    Lattice scaling: the larger of U_t = beta Re_x nu / R_c and the buoyancy
    velocity U_b = sqrt(g beta dT R_c) = nu sqrt(Gr) / R_c is set to u_ref, so
    that the flow stays at low Mach number whichever force drives it."""
    rc = float(nr)
    nu = u_ref * rc / max(beta * re_x, math.sqrt(grashof) if grashof > 0.0 else 0.0)
    omega_x = re_x * nu / (rc * rc)
    omega_c = re_c_ratio * re_x * nu / (rc * rc)
    tau = 3.0 * nu + 0.5
    kappa = nu / prandtl
    tau_t = 2.0 * kappa + 0.5
    gbeta = grashof * nu * nu / rc ** 3
    return Problem(nr=nr, nz=nr, tau=tau, rho0=rho0, z_lo=WALL, z_hi=MIXED, swirl=True,
                   temperature=True, tau_t=tau_t, gbeta=gbeta, t_ref=0.5,
                   r_split=beta * rc,
                   omega={"outer": omega_c, "lo": omega_c, "hi": omega_x},
                   t_wall={"outer": 1.0, "hi": 0.0}, collision=collision,
                   name=f"wheeler Re_x={re_x:g} Pr={prandtl:g} Gr={grashof:.3g} {nr}x{nr}")


def large_pipe(nr: int = 4096, nz: int = 8192, tau: float = 0.8, umax: float = 0.01) -> Problem:
    """Large Hagen-Poiseuille pipe (D2Q9 only), sized well beyond the L2 cache."""
    p = hagen_poiseuille(nr=nr, nz=nz, tau=tau, umax=umax)
    p.name = f"pipe {nr}x{nz}"
    return p


def batch_sweep(seed: int = 20261202, n_cavities: int = 256, n_wheeler: int = 64,
                scale: float = 1.0, collision: str = "mrt") -> List[Problem]:
    """Uneven batch: rotating-lid cavities with N_r ~ U{64..256}, H/R ~ U[1, 3.5],
    Re ~ U[500, 3000], plus Wheeler-type 128x128 cells with Pr alternating
    0.05 / 5, log10 Gr ~ U[4, 6], Re_x ~ U[100, 1000], Re_c = -Re_x / 4.
    ``scale`` shrinks every radius (for small test batches).  The high-Re draws
    reach tau_s ~ 0.506, the low-viscosity regime where the paper's BGK scheme
    is unstable (Sec. IV B); the sweep therefore uses its MRT scheme."""
    rng = np.random.default_rng(seed)
    out: List[Problem] = []
    for _ in range(n_cavities):
        nr = int(rng.integers(64, 257))
        aspect = float(rng.uniform(1.0, 3.5))
        re = float(rng.uniform(500.0, 3000.0))
        nr_s = max(4, int(round(nr * scale)))
        out.append(rotating_lid_cavity(nr=nr_s, aspect=aspect, re=re, collision=collision))
    for i in range(n_wheeler):
        pr = 0.05 if i % 2 == 0 else 5.0
        gr = 10.0 ** float(rng.uniform(4.0, 6.0))
        re_x = float(rng.uniform(100.0, 1000.0))
        nr_s = max(4, int(round(128 * scale)))
        out.append(wheeler_cell(nr=nr_s, re_x=re_x, prandtl=pr, grashof=gr, collision=collision))
    return out


# ----------------------------------------------------------------------------- warm-start inputs


def warm_start_geometry(pb: Problem) -> Dict[str, float]:
    """Where a Problem sits on the warm-start canvas: radius of column 0 and of
    the side wall (canvas r = 1), height of row 0, of the bottom wall (canvas
    z = 0) and the bottom-to-top distance (canvas z = 1), and the velocity
    scale (the lid's speed at the side wall)."""
    z_first = 0.0 if pb.z_lo == NEE else 0.5
    z_top = (pb.nz - 1) + z_first + (0.0 if pb.z_hi == NEE else 0.5)
    r_wall = pb.wall_radius
    return dict(r_first=float(pb.node_radius(0)), r_wall=r_wall, z_first=z_first, z_bottom=0.0, height=z_top,
                u_scale=pb.omega_of("hi") * r_wall)


def warm_start_features(pb: Problem) -> List[float]:
    """The six features of a Problem for the warm-start network: kind (0 cavity,
    1 Wheeler-type cell), H/R / 3.5, log10(Re) - 3 with Re = Omega_lid R^2 / nu,
    log10(1 + Gr) / 6 with Gr = g beta R^3 / nu^2 (dT = 1), log10(Pr) / 2, and
    Omega_side / Omega_lid."""
    g = warm_start_geometry(pb)
    radius = g["r_wall"]
    nu = (pb.tau - 0.5) / 3.0
    om = pb.omega_of("hi")
    re = abs(om) * radius * radius / nu if om != 0.0 else 1.0
    kind = 1.0 if (pb.temperature or pb.z_hi == MIXED) else 0.0
    gr = pb.gbeta * radius ** 3 / nu ** 2 if pb.temperature else 0.0
    pr = nu / ((pb.tau_t - 0.5) / 2.0) if pb.temperature else 1.0
    ratio = pb.omega_of("outer") / om if om != 0.0 else 0.0
    return [kind, g["height"] / radius / 3.5, math.log10(re) - 3.0, math.log10(1.0 + max(gr, 0.0)) / 6.0,
            math.log10(pr) / 2.0, ratio]


# ----------------------------------------------------------------------------- random fields


def random_fields(nr: int, nz: int, seed: int, rho0: float = 1.0, drho: float = 1e-2,
                  du: float = 1e-2, duth: float = 1e-2, t_mean: float = 0.5,
                  dt: float = 0.2) -> np.ndarray:
    """Seeded smooth random macroscopic fields, shape [5][nz][nr] float64:
    rho, u_r, u_z, u_theta, T.  A few random Fourier modes plus small noise."""
    rng = np.random.default_rng(seed)
    j = (np.arange(nr) + 0.5) / max(nr, 1)
    k = (np.arange(nz) + 0.5) / max(nz, 1)
    zz, rr = np.meshgrid(k, j, indexing="ij")
    out = np.empty((5, nz, nr), dtype=np.float64)
    amps = (drho, du, du, duth, dt)
    for q in range(5):
        acc = np.zeros((nz, nr))
        for _ in range(4):
            kr, kz = rng.integers(1, 4, size=2)
            ph = rng.uniform(0.0, 2.0 * np.pi, size=2)
            acc += rng.uniform(-1.0, 1.0) * np.sin(np.pi * kr * rr + ph[0]) * np.cos(np.pi * kz * zz + ph[1])
        acc += 0.25 * rng.uniform(-1.0, 1.0, size=(nz, nr))
        acc /= max(np.max(np.abs(acc)), 1e-300)
        out[q] = amps[q] * acc
    out[0] += rho0
    out[4] += t_mean
    return out


def random_noise(shape, seed: int, amplitude: float) -> np.ndarray:
    """Seeded multiplicative noise 1 + amplitude * U[-1, 1]."""
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=shape)
