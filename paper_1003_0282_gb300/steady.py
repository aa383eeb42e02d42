"""Running domains to a steady state, with a JSON-lines progress log.

A domain is steady when the residual of Eq. 57 (the largest change of the
in-plane speed per step, between two consecutive levels or, with the
solver's residual lag 2, across two levels) is at or below a tolerance.
run_to_steady advances a Batch (or a single Domain) in calls of `chunk`
lattice steps.  Each call ends with the library's two check steps, which
give every domain's residual, mass and mass budget.  The run records when
each domain first reaches the tolerance, marks domains whose check values
became non-finite, and stops when no domain is left to wait for or after
max_steps.  With a log, every call appends one JSON line: time level, steps,
wall seconds, the call's MLUPS, the largest finite residual, counts of
converged and blown-up domains, and the summed mass and budget.

Host logic only: every lattice step runs in the CUDA library.
"""
from __future__ import annotations

import json
import time
from typing import IO, Optional

import numpy as np


def check_values(solver) -> np.ndarray:
    """[n][3] residual, mass and budget of the last check step (non-finite allowed)."""
    if hasattr(solver, "residuals"):
        return np.asarray(solver.residuals(allow_nonfinite=True), dtype=np.float64).reshape(-1, 3)
    return np.asarray([solver.residual(allow_nonfinite=True)], dtype=np.float64)


def problems_of(solver) -> list:
    problems = getattr(solver, "problems", None)
    return list(problems) if problems is not None else [solver.pb]


def run_to_steady(solver, tol: float, max_steps: int, chunk: int = 5000, log: Optional[IO[str]] = None,
                  t0: Optional[float] = None) -> dict:
    """Step `solver` until every domain is steady (residual <= tol) or blown up, or max_steps ran.

    t0 is the time.perf_counter() value the wall times count from (default:
    the call).  Returns reached (int64 [n]: steps when the domain first met
    tol, -1 if never), when (float [n]: seconds since t0, NaN if never),
    blown (bool [n]: mass became non-finite) and steps (lattice steps run).
    """
    if chunk < 3:
        raise ValueError("chunk must be >= 3 (each call ends with its check steps)")
    t0 = time.perf_counter() if t0 is None else t0
    problems = problems_of(solver)
    n, nodes = len(problems), int(sum(p.cells for p in problems))
    reached = np.full(n, -1, dtype=np.int64)
    blown = np.zeros(n, dtype=bool)
    when = np.full(n, np.nan)
    steps = 0
    last = time.perf_counter()
    while steps < max_steps and np.any((reached < 0) & ~blown):
        solver.step(chunk)
        steps += chunk
        vals = check_values(solver)  # synchronises
        if vals.shape[0] != n:
            raise ValueError(f"{vals.shape[0]} check values for {n} domains")
        now_abs = time.perf_counter()
        now = now_abs - t0
        res = vals[:, 0]
        newly = (reached < 0) & (res <= tol) & np.isfinite(res)
        reached[newly] = steps
        when[newly] = now
        blown |= ~np.isfinite(vals[:, 1])
        if log is not None:
            finite = np.isfinite(res)
            ok = np.isfinite(vals[:, 1])
            log.write(json.dumps({
                "t": int(solver.time), "steps": steps, "wall_s": now,
                "mlups": nodes * chunk / max(now_abs - last, 1e-12) / 1e6,
                "residual_max": float(res[finite].max()) if finite.any() else None,
                "converged": int((reached >= 0).sum()), "blown": int(blown.sum()), "domains": n,
                "mass": float(vals[ok, 1].sum()), "budget": float(vals[ok, 2].sum()),
            }) + "\n")
            log.flush()
        last = now_abs
    return dict(reached=reached, when=when, blown=blown, steps=steps)


def _main(argv=None) -> int:
    """Run one rotating-lid cavity (Sec. IV B) from rest to the Eq. 57
    criterion and save its fields; with --against, print the per-field
    difference from a saved run (the FP64 one) over the lid speed."""
    import argparse

    from . import axlbm as B
    from . import inputs as I

    p = argparse.ArgumentParser(prog="python -m paper_1003_0282_gb300.steady")
    p.add_argument("--cavity", nargs=3, type=float, metavar=("NR", "ASPECT", "RE"), required=True)
    p.add_argument("--collision", default="mrt", choices=["bgk", "mrt"])
    p.add_argument("--precision", default="fp32", choices=sorted(B.PRECISIONS))
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--lag", type=int, default=2, choices=[1, 2])
    p.add_argument("--max-steps", type=int, default=10_000_000)
    p.add_argument("--chunk", type=int, default=20_000)
    p.add_argument("--log", default=None, help="JSON-lines progress log")
    p.add_argument("--save", default=None, help=".npz of rho, u_r, u_z, u_theta and the run's record")
    p.add_argument("--against", default=None, help="a saved run to compare with")
    a = p.parse_args(argv)
    nr = int(a.cavity[0])
    pb = I.rotating_lid_cavity(nr=nr, aspect=a.cavity[1], re=a.cavity[2], collision=a.collision)
    lid = pb.omega_of("hi") * pb.wall_radius
    dom = B.Domain(pb, a.precision)
    dom.set_residual_lag(a.lag)
    log = open(a.log, "a") if a.log else None
    try:
        out = run_to_steady(dom, a.tol, a.max_steps, chunk=a.chunk, log=log)
    finally:
        if log:
            log.close()
    res, mass, budget = dom.residual(allow_nonfinite=True)
    fields = dom.moments(B.RHO | B.UR | B.UZ | B.UTH)
    dom.close()
    rec = {"problem": pb.name, "precision": a.precision, "collision": a.collision, "tol": a.tol, "lag": a.lag,
           "steps": int(out["steps"]), "reached": int(out["reached"][0]), "wall_s": float(out["when"][0]),
           "residual": float(res), "mass": float(mass), "lid_speed": float(lid)}
    if a.against:
        ref = np.load(a.against)
        want = ref["fields"]
        rec["against"] = {"run": str(ref["precision"]), "steps": int(ref["steps"]),
                          "max_error_over_lid_speed": {
                              name: float(np.max(np.abs(fields[q] - want[q]))) / (lid if q else 1.0)
                              for q, name in enumerate(("rho", "u_r", "u_z", "u_theta"))}}
    if a.save:
        np.savez_compressed(a.save, fields=fields, precision=a.precision, steps=out["steps"],
                            record=json.dumps(rec))
    print(json.dumps(rec), flush=True)
    return 0 if out["reached"][0] >= 0 else 1


if __name__ == "__main__":
    raise SystemExit(_main())
