"""Shared helpers of the GPU parity tests (imported by test modules only).

Initial states are built on the oracle side from the seeded generators and
uploaded through the C ABI; expected values always come from the oracle.
"""
import dataclasses

import numpy as np

import oracle
from paper_1003_0282_gb300 import inputs as I

# Storage precision -> relative max-norm tolerance on populations after N steps.
# FP64: 1e-10 and FP32: 1e-5 as the design targets state; the 16-bit modes
# are measured per field elsewhere.
POP_TOL = {"fp64": 1e-10, "fp32": 1e-5}

BOUNDARY_MIXES = {
    "pipe": dict(inner="axis", z_lo="periodic", z_hi="periodic"),
    "closed": dict(inner="axis", z_lo="wall", z_hi="wall"),
    "free-top": dict(inner="axis", z_lo="wall", z_hi="free"),
    "crystal": dict(inner="axis", z_lo="wall", z_hi="mixed", r_split=0.4),  # r_split scaled by nr below
    "annulus-mixed": dict(inner="wall", r0=5.0, z_lo="wall", z_hi="mixed", r_split=0.5),
    "annulus-pipe": dict(inner="wall", r0=2.0, z_lo="periodic", z_hi="periodic"),
    # node on the axis (Sec. IV A)
    "axis-node-pipe": dict(inner="axis_node", z_lo="periodic", z_hi="periodic"),
    "axis-node-crystal": dict(inner="axis_node", z_lo="wall", z_hi="mixed", r_split=0.4),
    "axis-node-free-top": dict(inner="axis_node", z_lo="free", z_hi="free"),
    # wet walls (non-equilibrium extrapolation, Sec. IV B)
    "nee-cavity": dict(inner="axis", outer="nee", z_lo="nee", z_hi="nee"),
    "nee-axis-node": dict(inner="axis_node", outer="nee", z_lo="nee", z_hi="mixed", r_split=0.4),
    "nee-annulus-pipe": dict(inner="wall", r0=3.0, outer="nee", z_lo="periodic", z_hi="periodic"),
    # Zou-He pipe wall (Sec. IV A; D2Q9 only)
    "zou-he-pipe": dict(inner="axis_node", outer="zou_he", z_lo="periodic", z_hi="periodic"),
}


def problem(nr, nz, mix, swirl=True, temperature=True, tau=0.8, collision="bgk", **extra):
    kw = dict(BOUNDARY_MIXES[mix])
    if kw.get("outer") == "zou_he":  # a Zou-He pipe carries f only
        swirl = temperature = False
    if "r_split" in kw:
        kw["r_split"] = kw["r_split"] * nr + kw.get("r0", 0.0)
    kw.update(extra)
    return I.Problem(nr=nr, nz=nz, tau=tau, swirl=swirl, temperature=temperature, tau_t=0.7,
                     az0=2e-6, omega_t=0.003, gbeta=3e-4, t_ref=0.5, rho0=1.0,
                     omega={"inner": 0.001, "outer": 0.002, "lo": -0.001, "hi": 0.003},
                     t_wall={"outer": 1.0, "hi": 0.0}, collision=collision, **kw)


def seeded_state(pb, seed):
    """Oracle-side initial state: equilibria of seeded random fields, perturbed."""
    fields = I.random_fields(pb.nr, pb.nz, seed=seed)
    st = oracle.equilibrium(pb, fields)
    st.f *= I.random_noise(st.f.shape, seed=seed + 1, amplitude=0.01)
    st.g *= I.random_noise(st.g.shape, seed=seed + 2, amplitude=0.05)
    st.h *= I.random_noise(st.h.shape, seed=seed + 3, amplitude=0.01)
    return st


def rel_err(got, want):
    scale = max(float(np.max(np.abs(want))), 1e-300)
    return float(np.max(np.abs(got - want))) / scale


def upload(dom, st):
    dom.set_populations(st.f, st.g if st.pb.swirl else None, st.h if st.pb.temperature else None, time=st.t)


def compare_populations(dom, st):
    f, g, h = dom.get_populations()
    errs = {"f": rel_err(f, st.f)}
    if st.pb.swirl:
        errs["g"] = rel_err(g, st.g)
    if st.pb.temperature:
        errs["h"] = rel_err(h, st.h)
    return errs


def window_oracle(pops, pb, j0, k0, steps, t0):
    """Oracle prediction of the populations of node (j0, k0) after `steps` steps,
    from the full-domain populations `pops` = (f, g, h) at time t0.

    A window of half-width `steps` around the node is advanced by the oracle.
    Where the window reaches a physical boundary the window uses it; its other
    edges (and a periodic wrap) only corrupt nodes within `steps` of those
    edges, which the centre node never sees.  A wet wall rebuilds its nodes
    from the next two nodes inwards, so information travels two nodes
    further; the window has that margin."""
    f, g, h = pops
    s = steps + 2
    ja, jb = max(0, j0 - s), min(pb.nr, j0 + s + 1)
    inner = pb.inner if ja == 0 else "wall"
    # a window away from the axis is an annulus with the same node radii
    r0 = pb.r0 + ja - (0.5 if (pb.inner == "axis_node" and ja > 0) else 0.0)
    # z rows (periodic domains wrap; walls clip)
    if pb.z_lo == "periodic":
        rows = [(k0 + d) % pb.nz for d in range(-s, s + 1)] if pb.nz >= 2 * s + 1 else list(range(pb.nz))
        z_lo = z_hi = "periodic"
        kc = s if pb.nz >= 2 * s + 1 else k0
    else:
        ka, kb = max(0, k0 - s), min(pb.nz, k0 + s + 1)
        rows = list(range(ka, kb))
        z_lo = pb.z_lo if ka == 0 else "wall"
        z_hi = pb.z_hi if kb == pb.nz else "wall"
        kc = k0 - ka
    outer = pb.outer if jb == pb.nr else "wall"
    sub = dataclasses.replace(pb, nr=jb - ja, nz=len(rows), inner=inner, r0=r0, z_lo=z_lo, z_hi=z_hi, outer=outer)
    cut = lambda a: None if a is None else np.ascontiguousarray(a[:, rows, ja:jb])
    st = oracle.State(sub, cut(f), cut(g), cut(h), t=t0)
    oracle.step(st, steps)
    jc = j0 - ja
    return st.f[:, kc, jc], (st.g[:, kc, jc] if pb.swirl else None), (st.h[:, kc, jc] if pb.temperature else None)


def record(filename, name, value):
    """Merge `value` under `name` into the JSON file `filename` of the
    directory named by the AXLBM_TEST_RECORD environment variable (measured
    values the tests see, for reports); nothing is written when it is unset."""
    import json
    import os
    folder = os.environ.get("AXLBM_TEST_RECORD")
    if not folder:
        return
    os.makedirs(folder, exist_ok=True)
    path = os.path.join(folder, filename)
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    data[name] = value
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1)
