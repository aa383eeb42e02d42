"""Throughput benchmark of the axisymmetric lattice Boltzmann hot path.

One benchmark step = one solver call of --inner lattice time steps over the
whole workload (bulk collide-and-stream, boundary rings, and the check step
with its FP64 reductions that ends every call).  The metric is MLUPS:
million lattice-node updates per second, whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch|pipe] [--precision fp32|fp16|...]

Default workload (``batch``): the uneven sweep -- 256 rotating-lid cavities
(N_r ~ U{64..256}, H/R ~ U[1, 3.5], Re ~ U[500, 3000]) and 64 Wheeler-type
128 x 128 cells with temperature (Pr 0.05 / 5, Gr 1e4-1e6), 17.0 M nodes, one
persistent launch per step, FP32 arithmetic and FP32 deviation storage
(1.5 GB, far larger than the 129 MB L2, so no cache flush is needed).
``pipe``: one 4096 x 8192 Hagen-Poiseuille pipe (D2Q9 only).  Under torchrun
every rank advances its own seeded sweep (independent domains, no collective
on the data path): weak scaling.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM traffic of the bulk kernel from the ncu capture summarised in profiles/:
# (dram__bytes_read.sum + dram__bytes_write.sum) / algorithmic bytes of the
# captured launch, keyed by kernel and the SHA-256 prefix of the kernel source
# at capture time.  Reported as null once the source has changed.
NCU_TRAFFIC = {
    # profiles/k_bulk_batch_fp32_sweep320_launches.md: one even and one odd launch (4 x 128 tiles)
    "batch fp32": {"src_sha": "9953980fb660c4fe", "dram_per_alg_byte": 0.9899},
    # profiles/k_bulk_batch_fp16_sweep_half_full.md: full-size DRAM capture, one even (8 x 128) and one odd launch
    "batch fp16": {"src_sha": "9953980fb660c4fe", "dram_per_alg_byte": 0.9657},
    # profiles/k_bulk_fp32_pipe4096x8192_launches.md: one even and one odd launch (4 x 128 tiles)
    "pipe fp32": {"src_sha": "9953980fb660c4fe", "dram_per_alg_byte": 1.0577},
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--inner", type=int, default=50, help="lattice time steps per benchmark step")
    p.add_argument("--workload", choices=["batch", "pipe", "warmstart"], default="batch",
                   help="warmstart: time to a steady state from rest and from the warm-start network")
    p.add_argument("--scale", type=float, default=1.0, help="batch: shrink every domain (small profiling cases)")
    p.add_argument("--tile", default=None,
                   help="batch: bulk tile shape RxN for both steps, or RxN,RxN for even and odd steps, instead "
                        "of the timed ones (4x128 or 8x64; also 8x128 with FP16 storage)")
    p.add_argument("--nr", type=int, default=4096)
    p.add_argument("--nz", type=int, default=8192)
    p.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16", "bf16"])
    p.add_argument("--e2e-steps", type=int, default=8)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tol", type=float, default=1e-8,
                   help="warmstart: per-domain residual (Eq. 57, across two levels) of a steady state")
    p.add_argument("--max-steps", type=int, default=2000000, help="warmstart: give up after this many steps")
    p.add_argument("--ws-seed", type=int, default=20, help="warmstart: seed of the held-out draws")
    p.add_argument("--ws-draws", type=int, default=200, help="warmstart: held-out draws")
    p.add_argument("--metrics-log", default=None,
                   help="warmstart: write one JSON line per 5000 steps to PREFIX.rest.jsonl / PREFIX.warm.jsonl")
    p.add_argument("--shard", choices=["weak", "strong"], default="weak",
                   help="batch under torchrun: a sweep per rank (weak) or one sweep split over the ranks (strong)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for name in ("ops_impl.cuh", "lattice.cuh", "pair.cuh", "tma.cuh", "batch.cuh", "batch.cu", "batch_ops.cuh",
                 "batch_internal.h"):
        with open(os.path.join(ROOT, "paper_1003_0282_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_sample(workload: str):
    """A bounded piece of the workload for the oracle: one rotating-lid cavity
    of the sweep's kind, 128 x 192 (the smallest grid of the cavity family),
    for the batch, or a 256 x 512 pipe section for the pipe."""
    from paper_1003_0282_gb300 import inputs as I
    if workload == "pipe":
        return I.hagen_poiseuille(nr=256, nz=512, tau=0.8, umax=0.01), "pipe section 256x512"
    return I.rotating_lid_cavity(nr=128, aspect=1.5, re=990.0), "rotating-lid cavity 128x192 (A 1.5, Re 990)"


def host_cpu() -> dict:
    """Model name and logical core count of the host the CPU legs run on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu": model or platform.machine(), "host_cores": os.cpu_count()}


def oracle_configs():
    """The oracle's single-thread samples beside the GPU workload: the pipe,
    Womersley and cavity configurations (the smallest grid of the cavity
    family) and a 256 x 512 cavity."""
    from paper_1003_0282_gb300 import inputs as I
    return [("Hagen-Poiseuille pipe 32x8", I.hagen_poiseuille(nr=32, nz=8, tau=0.8, umax=0.01)),
            ("Womersley pipe 64x4 (alpha 5)", I.womersley(nr=64, nz=4, tau=0.8, alpha=5.0)),
            ("rotating-lid cavity 128x192 (A 1.5, Re 990)", I.rotating_lid_cavity(nr=128, aspect=1.5, re=990.0)),
            ("rotating-lid cavity 256x512 (A 2, Re 990)", I.rotating_lid_cavity(nr=256, aspect=2.0, re=990.0))]


def cpu_baseline(workload: str, inner: int, budget_s: float = 16.0):
    """The FP64 oracle, as it stands, single-threaded, on bounded samples:
    ~budget_s / 4 of CPU time on each of oracle_configs() (the pipe workload
    times its 256 x 512 pipe section instead of the cavities).  `value` is the
    128 x 192 cavity's (the pipe section's for the pipe workload)."""
    import oracle

    samples = oracle_configs()
    if workload == "pipe":
        samples = samples[:2] + [cpu_sample("pipe")[::-1]]
    per = {}
    for what, sample in samples:
        st = oracle.rest_state(sample)
        oracle.step(st, 2)
        steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s / len(samples):
            oracle.step(st, inner)
            steps += inner
        dt = time.perf_counter() - t0
        per[what] = {"MLUPS": sample.cells * steps / dt / 1e6, "steps": steps, "seconds": round(dt, 2)}
    main = samples[2][0]
    return {"value": per[main]["MLUPS"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle, single thread: {main} (value) and the other configurations below, "
                      f"~{budget_s / len(samples):.0f} s each", "configs": per, **host_cpu()}


def workload_name(args, problems):
    """The workload of a run (the same text for both arms)."""
    if args.workload == "pipe":
        pb = problems[0]
        return f"pipe {pb.nr}x{pb.nz} D2Q9 (Hagen-Poiseuille force, axis + bounce-back wall, periodic z)"
    return (f"batched uneven sweep: {sum(not p.temperature for p in problems)} rotating-lid cavities + "
            f"{sum(p.temperature for p in problems)} Wheeler-type cells with temperature, one persistent "
            f"launch per step" + (f" (radii scaled by {args.scale})" if args.scale != 1.0 else ""))


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, one bounded
    sample of the workload per benchmark step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1003_0282_gb300 import inputs as I

    sample, what = cpu_sample(args.workload)
    st = oracle.rest_state(sample)
    inner = max(1, min(args.inner, 10))
    for _ in range(args.warmup):
        oracle.step(st, inner)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(st, inner)
    dt = time.perf_counter() - t0
    value = sample.cells * inner * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, [I.large_pipe(nr=args.nr, nz=args.nz)] if args.workload == "pipe"
                                             else I.batch_sweep(scale=args.scale)),
                   "precision": "fp64 oracle", "sample": f"{what}, {inner} lattice steps per benchmark step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{what} x {inner} lattice steps per benchmark step", **host_cpu()},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def heldout_draws(seed: int, scale: float, count: int):
    """`count` held-out draws of the uneven sweep's distribution (seed `seed`),
    cavities and Wheeler-type cells in the sweep's 4 : 1 proportion."""
    from paper_1003_0282_gb300 import inputs as I

    sweep = I.batch_sweep(seed=seed, scale=scale)
    cav = [p for p in sweep if not p.temperature]
    whe = [p for p in sweep if p.temperature]
    nw = max(1, round(count / 5)) if count > 1 else 0
    return cav[:count - nw] + whe[:nw]


def run_warmstart(args):
    """Steps and wall time until each domain of a held-out set of draws
    reaches a steady state (residual of Eq. 57, measured across two levels,
    <= tol), from rest and from the fields of the warm-start network (its
    inference and the initialisation inside the timed region).  Domains that
    converge in neither arm within max_steps are reported and left out of
    both."""
    import torch
    from paper_1003_0282_gb300 import axlbm as B
    from paper_1003_0282_gb300 import inputs as I
    from paper_1003_0282_gb300 import steady

    path = os.path.join(ROOT, "paper_1003_0282_gb300", "warm_start_weights.npz")
    if not os.path.exists(path):
        print(json.dumps({"workload": "warmstart", "unavailable": "no trained weights (run warm_start_train)"}))
        return
    weights = np.load(path)["weights"]
    probs = heldout_draws(args.ws_seed, args.scale, args.ws_draws)
    arms = {}
    for arm in ("rest", "warm"):
        batch = B.Batch(probs, "fp32")
        batch.set_residual_lag(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if arm == "warm":
            ws = B.WarmStart(weights)
            ws.start(batch, probs)
            ws.close()
        log = open(f"{args.metrics_log}.{arm}.jsonl", "w") if args.metrics_log else None
        run = steady.run_to_steady(batch, args.tol, args.max_steps, chunk=5000, log=log, t0=t0)
        if log:
            log.close()
        uz = [batch.moments(d, B.UZ, dtype=np.float32)[0] for d in range(len(probs))]
        batch.close()
        arms[arm] = dict(reached=run["reached"], when=run["when"], blown=run["blown"], uz=uz, steps=run["steps"])
    rest, warm = arms["rest"], arms["warm"]
    both = (rest["reached"] > 0) & (warm["reached"] > 0)
    n_ok = int(both.sum())
    out = {}
    for arm in ("rest", "warm"):
        a = arms[arm]
        out[arm] = dict(converged=int((a["reached"] > 0).sum()), blown=int(a["blown"].sum()),
                        steps_median=float(np.median(a["reached"][both])) if n_ok else None,
                        steps_max=int(a["reached"][both].max()) if n_ok else None,
                        time_median_s=float(np.median(a["when"][both])) if n_ok else None,
                        time_all_s=float(np.max(a["when"][both])) if n_ok else None,
                        steps_run=int(a["steps"]))
    # the steady fields of the two arms at the end of the run, where both are finite
    lid = np.array([I.warm_start_geometry(p)["u_scale"] for p in probs])
    difs = np.array([float(np.max(np.abs(rest["uz"][d] - warm["uz"][d]))) / abs(lid[d])
                     if both[d] and np.all(np.isfinite(rest["uz"][d])) and np.all(np.isfinite(warm["uz"][d]))
                     else np.nan for d in range(len(probs))])
    fin = np.isfinite(difs)
    excluded = {"not_converged_in_either_arm": int(np.sum((rest["reached"] < 0) & (warm["reached"] < 0))),
                "converged_in_one_arm_only": int(np.sum((rest["reached"] > 0) != (warm["reached"] > 0))),
                "blown_up_in_either_arm": int(np.sum(rest["blown"] | warm["blown"]))}
    ratio = lambda a, b: (a / b) if (a is not None and b) else None
    line = {
        "metric": "time_to_steady_median", "value": out["warm"]["time_median_s"], "unit": "s",
        "higher_is_better": False,
        "n_gpus": 1, "dtype": "f32", "data": "synthetic", "vs_baseline": None,
        "config": {"workload": f"{len(probs)} held-out draws of the uneven sweep (seed {args.ws_seed}, radii "
                               f"x{args.scale}), from rest and from the warm-start network, to the Eq. 57 residual "
                               f"<= {args.tol:g} measured across two levels, at most {args.max_steps} steps",
                   "rest": out["rest"], "warm_start": out["warm"], "converged_in_both": n_ok,
                   "excluded": excluded,
                   "steady_uz_difference_over_lid_speed": {
                       "max": float(np.max(difs[fin])) if fin.any() else None,
                       "median": float(np.median(difs[fin])) if fin.any() else None, "domains": int(fin.sum())},
                   "speedup_steps_median": ratio(out["rest"]["steps_median"], out["warm"]["steps_median"]),
                   "speedup_time_median": ratio(out["rest"]["time_median_s"], out["warm"]["time_median_s"]),
                   "speedup_time_all": ratio(out["rest"]["time_all_s"], out["warm"]["time_all_s"])},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "warmstart":
        run_warmstart(args)
        return
    import torch
    import torch.distributed as dist

    if not torch.cuda.is_available():
        sys.exit("bench.py: no CUDA device; the solver runs only in the CUDA library (there is no CPU path)")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_1003_0282_gb300 import axlbm as B
    from paper_1003_0282_gb300 import inputs as I
    from paper_1003_0282_gb300 import shard as S

    if args.workload == "pipe":
        pb = I.large_pipe(nr=args.nr, nz=args.nz)
        problems = [pb]
        solver = B.Domain(pb, args.precision)
        solver.set_fields(torch.tensor(I.random_fields(pb.nr, pb.nz, seed=1000 + rank, du=1e-3, duth=0.0),
                                       dtype=torch.float32, device="cuda"))
        timing_on = lambda on: B.axlbm_kernel_timing(solver.handle, on)
        kernel_times = lambda: B.axlbm_kernel_times(solver.handle)
        parity_times = None
        tile = (4, 128)
        workload = workload_name(args, [pb])
    else:
        problems = S.rank_problems(I.batch_sweep, world, rank, args.shard, scale=args.scale)
        solver = B.Batch(problems, args.precision)
        timing_on = lambda on: B.axlbm_batch_kernel_timing(solver.handle, on)
        kernel_times = lambda: B.axlbm_batch_kernel_times(solver.handle)
        parity_times = lambda: B.axlbm_batch_kernel_times_by_parity(solver.handle)
        if args.tile:
            shapes = [tuple(int(v) for v in t.split("x")) for t in args.tile.split(",")]
            solver.tile_shapes = (shapes[0], shapes[-1])
        tile = solver.tile_shapes
        workload = workload_name(args, problems)
    nodes = sum(p.cells for p in problems)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.step(args.inner)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            solver.step(args.inner)
        ev1.record(stream)
        barrier()
        # the kernel times: the same steps again with the library's events
        # around every bulk launch (which launches kernel by kernel)
        timing_on(True)
        for _ in range(args.steps):
            solver.step(args.inner)
        barrier()
        bulk_n, bulk_ms, bulk_bytes, all_launches = kernel_times()
        by_parity = parity_times() if parity_times else None
        timing_on(False)
    ms = ev0.elapsed_time(ev1)
    caps, glaunch = solver.graph_stats()
    graphs = (f"plain step pairs from captured CUDA graphs ({glaunch} graph launches, {caps} captures)"
              if glaunch else "kernel by kernel")
    if args.workload == "pipe":
        res, mass, _ = solver.residual()
    else:
        rr = solver.residuals()
        res, mass = float(rr[:, 0].max()), float(rr[:, 1].sum())
    ms = S.max_over_ranks(ms)
    res = S.max_over_ranks(res)
    mass = S.sum_over_ranks(mass)
    all_nodes = int(round(S.sum_over_ranks(nodes)))
    updates = all_nodes * args.inner * args.steps
    value = updates / (ms / 1e3) / 1e6

    # end to end through the C ABI with pinned host buffers: fields in, moments out
    fin = np.concatenate([I.random_fields(p.nr, p.nz, seed=2000 + rank + i, du=1e-3, duth=1e-3).ravel()
                          for i, p in enumerate(problems)])
    host_in = torch.empty(fin.size, dtype=torch.float32, pin_memory=True)
    host_in.copy_(torch.from_numpy(fin.astype(np.float32)))
    host_out = torch.empty(3 * nodes, dtype=torch.float32, pin_memory=True)
    if solver.time % 2:
        solver.step(1)  # fields are set at an even level
    if args.workload != "pipe":  # the copy streams and their staging buffers are made by the first call
        B.axlbm_batch_set_fields_all_async(solver.handle, host_in.data_ptr(), B.F32)
        B.axlbm_batch_moments_all_async(solver.handle, B.RHO | B.UR | B.UZ, host_out.data_ptr(), B.F32)
        B.axlbm_batch_set_fields_all_async(solver.handle, host_in.data_ptr(), B.F32)
        B.axlbm_batch_moments_all_async(solver.handle, B.RHO | B.UR | B.UZ, host_out.data_ptr(), B.F32)
        B.axlbm_batch_sync(solver.handle)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        if args.workload == "pipe":
            B.axlbm_set_fields(solver.handle, host_in.data_ptr(), B.F32, 0)
            solver.step(args.inner)
            B.axlbm_moments(solver.handle, B.RHO | B.UR | B.UZ, host_out.data_ptr(), B.F32, 0)
        else:
            # copies on the batch's copy streams: this step's upload runs beside the previous step's
            # lattice steps, its download beside the next one's
            B.axlbm_batch_set_fields_all_async(solver.handle, host_in.data_ptr(), B.F32)
            solver.step(args.inner)
            B.axlbm_batch_moments_all_async(solver.handle, B.RHO | B.UR | B.UZ, host_out.data_ptr(), B.F32)
    if args.workload != "pipe":
        B.axlbm_batch_sync(solver.handle)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = S.max_over_ranks(e2e_s)
    e2e_value = all_nodes * args.inner * args.e2e_steps / e2e_s / 1e6
    solver.close()

    if rank == 0:
        peak, peak_kind = peaks()
        achieved = bulk_bytes / (bulk_ms / 1e3) / 1e9 if bulk_ms > 0 else 0.0
        sha = kernel_source_sha()
        key = f"{args.workload} {args.precision}"
        tr = NCU_TRAFFIC.get(key)
        traffic = None
        if tr and tr["src_sha"] == sha:
            traffic = tr["dram_per_alg_byte"] * bulk_bytes / max(bulk_n, 1)
        kernel = "k_bulk (even + odd AA steps)" if args.workload == "pipe" else "k_bulk_batch (even + odd AA steps)"
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": args.shard if (world > 1 and args.workload == "batch") else "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": workload, "precision": args.precision, "nodes": all_nodes,
                       "domains": len(problems), "lattice_steps_per_step": args.inner,
                       "bulk_tile": (f"{tile[0]}x{tile[1]}" if args.workload == "pipe" else
                                     f"{tile[0][0]}x{tile[0][1]} even, {tile[1][0]}x{tile[1][1]} odd"),
                       "launch": graphs,
                       "cache": "inputs larger than L2 (no flush)",
                       "parallelism": (f"independent domains on {world} ranks ({args.shard})" if world > 1
                                       else "one GPU")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": kernel, "launches": bulk_n,
                         "avg_launch_ms": bulk_ms / max(bulk_n, 1),
                         "alg_bytes_per_launch": bulk_bytes / max(bulk_n, 1)},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": 5 * 4 * all_nodes, "d2h_bytes_per_step": 3 * 4 * all_nodes,
                    "steps": args.e2e_steps,
                    "copies": ("synchronous, pinned host buffers" if args.workload == "pipe" else
                               "asynchronous on the batch's copy streams, pinned host buffers, one sync at the end")},
            "gpu_launches": all_launches,
            "clocks": clk.summary(),
            "check": {"residual": res, "mass": mass},
        }
        if by_parity:  # the even (in place) and odd (neighbour to neighbour) launches apart
            n2, ms2, by2 = by_parity
            line["roofline"]["by_parity"] = {
                name: {"launches": n2[p], "avg_launch_ms": ms2[p] / max(n2[p], 1),
                       "achieved": by2[p] / (ms2[p] / 1e3) / 1e9 if ms2[p] > 0 else 0.0}
                for p, name in enumerate(("even", "odd"))}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.inner)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
