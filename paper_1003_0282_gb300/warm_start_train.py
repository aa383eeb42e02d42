"""Train the warm-start network on solved draws of the uneven sweep.

    python -m paper_1003_0282_gb300.warm_start_train [--sweeps 10] [--scale 0.5]
        [--steps 1000000] [--iters 6000] [--out paper_1003_0282_gb300/warm_start_weights.npz]

Data: sweeps 1..S of ``inputs.batch_sweep`` (256 rotating-lid cavities and
64 Wheeler-type cells each, radii scaled by ``--scale``), each advanced from
rest by the batch solver for ``--steps`` lattice steps (draws that blow up
at the reduced resolution are dropped; the residual of Eq. 57 is measured
across two levels, which cancels the lattice's period-2 modes, and
reported); every domain's fields (u_r, u_z,
u_theta over the lid speed, T - T_ref) go onto the 256 (z) x 128 (r) canvas
with the library's resampling (``axlbm_ws_to_canvas``, the inverse of the
canvas-to-grid map).  The last sweep is held out.

Training runs in the library (``axlbm_ws_train_step``: forward and backward
kernels, BF16 implicit-GEMM convolutions on the tensor cores with FP32
accumulation, Adam on FP32 master weights) on
batches of 16 canvases with a cosine learning-rate schedule; PyTorch only
holds the device arrays.  The weights start from a uniform draw with bound
1/sqrt(fan_in) (kernels and biases) and are written as BF16 bit patterns in
the library's packing order (per layer: kernel [Cout][ky][kx][Cin], then bias).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_1003_0282_gb300 import axlbm as B  # noqa: E402
from paper_1003_0282_gb300 import inputs as I  # noqa: E402

# the library's network (include/axlbm.h): encoder levels 0-3, decoder levels 2, 1, 0, the 1x1 head
LAYERS = [(8, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 96, 3), (96, 96, 3), (96, 128, 3),
          (128, 128, 3), (224, 96, 3), (96, 96, 3), (160, 64, 3), (64, 64, 3), (96, 32, 3), (32, 32, 3),
          (32, 4, 1)]


def bf16_bits(x):
    """float -> BF16 bit patterns (round to nearest even), numpy uint16."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def initial_weights(seed):
    """Uniform weights and biases with bound 1/sqrt(fan_in), packed as the library expects."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, k in LAYERS:
        bound = 1.0 / math.sqrt(ci * k * k)
        parts.append(rng.uniform(-bound, bound, co * ci * k * k))
        parts.append(rng.uniform(-bound, bound, co))
    return bf16_bits(np.concatenate(parts))


def solve_sweep(ws, seed, scale, steps):
    """(features [n][6], canvases [n][4][256][128] on the device, residuals) of the finite draws."""
    import torch
    probs = I.batch_sweep(seed=seed, scale=scale)
    batch = B.Batch(probs, "fp32")
    batch.set_residual_lag(2)
    batch.step(steps)
    res = batch.residuals(allow_nonfinite=True)
    moms, keep = [], []
    for d, pb in enumerate(probs):
        if pb.temperature:
            m = batch.moments(d, B.UR | B.UZ | B.UTH | B.T, dtype=np.float32)
        else:  # no temperature: T = T_ref
            m3 = batch.moments(d, B.UR | B.UZ | B.UTH, dtype=np.float32)
            m = np.concatenate([m3, np.full((1,) + m3.shape[1:], pb.t_ref, dtype=np.float32)])
        if np.all(np.isfinite(m)):  # a draw that blew up (grid Reynolds number too high) is dropped
            moms.append(m.ravel())
            keep.append(d)
    batch.close()
    kept = [probs[d] for d in keep]
    canvas = ws.to_canvas(torch.tensor(np.concatenate(moms), device="cuda"), kept)
    feats = np.array([I.warm_start_features(pb) for pb in kept], dtype=np.float32)
    return feats, canvas, res[keep, 0]


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--scale", type=float, default=0.5)
    ap.add_argument("--steps", type=int, default=1000000)
    ap.add_argument("--iters", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "warm_start_weights.npz"))
    args = ap.parse_args()
    t0 = time.time()
    ws = B.WarmStart(initial_weights(args.seed))
    feats, canv, res = [], [], []
    for s in range(1, args.sweeps + 1):
        f, c, r = solve_sweep(ws, s, args.scale, args.steps)
        feats.append(f)
        canv.append(c)
        res.append(r)
        print(f"sweep {s}: {time.time() - t0:.0f} s, {len(f)} finite draws, residual median {np.median(r):.2e}, "
              f"<= 1e-8 in {int(np.sum(r <= 1e-8))}", flush=True)
    ftr = torch.tensor(np.concatenate(feats[:-1]), device="cuda")
    ctr = torch.cat(canv[:-1])
    fte, cte = torch.tensor(feats[-1], device="cuda"), canv[-1]
    g = torch.Generator(device="cpu").manual_seed(1)
    test = float("nan")
    for it in range(args.iters):
        idx = torch.randint(0, ftr.shape[0], (args.batch,), generator=g).to("cuda")
        lr = 0.5 * args.lr * (1.0 + math.cos(math.pi * it / args.iters))
        loss = ws.train_step(ftr.index_select(0, idx).contiguous(), ctr.index_select(0, idx).contiguous(), lr)
        if it % 500 == 0 or it == args.iters - 1:
            test = ws.loss(fte, cte)
            print(f"iter {it}: train {loss:.3e} held-out {test:.3e} ({time.time() - t0:.0f} s)", flush=True)
    bits = ws.weights()
    ws.close()
    assert bits.size == B.lib().axlbm_ws_weight_count()
    np.savez_compressed(args.out, weights=bits,
                        meta=json.dumps(dict(sweeps=args.sweeps, scale=args.scale, steps=args.steps, iters=args.iters,
                                             lr=args.lr, held_out_mse=test, trainer="axlbm_ws_train_step",
                                             train_draws=int(ftr.shape[0]), held_out_draws=int(fte.shape[0]),
                                             target_residual_median=float(np.median(np.concatenate(res))))))
    print(f"wrote {args.out} ({bits.size} weights), {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
