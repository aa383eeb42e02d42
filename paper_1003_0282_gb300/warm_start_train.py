"""Train the warm-start network on solved draws of the uneven sweep.

    python -m paper_1003_0282_gb300.warm_start_train [--sweeps 7] [--scale 0.5]
        [--steps 600000] [--iters 4000] [--out paper_1003_0282_gb300/warm_start_weights.npz]

Data: sweeps 1..S of ``inputs.batch_sweep`` (256 rotating-lid cavities and
64 Wheeler-type cells each, radii scaled by ``--scale``), each advanced from
rest by the batch solver for ``--steps`` lattice steps (draws that blow up
at the reduced resolution are dropped); every domain's
fields (u_r, u_z, u_theta over the lid speed, T - T_ref) are resampled onto
the 256 (z) x 128 (r) canvas -- the inverse of the library's canvas-to-grid
map (``axlbm_ws_fields``).  The last sweep is held out.

Model: the network of ``csrc/warmstart.cu`` written with PyTorch layers
(training only; inference runs in the library), Adam on the mean squared
error over the canvas, exported as BF16 bit patterns in the library's
packing order (per layer: kernel [Cout][ky][kx][Cin], then bias).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_1003_0282_gb300 import axlbm as B  # noqa: E402
from paper_1003_0282_gb300 import inputs as I  # noqa: E402

H, W = B.WS_CANVAS
LAYERS = [(8, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 128, 3), (128, 128, 3), (192, 64, 3),
          (64, 64, 3), (96, 32, 3), (32, 32, 3), (32, 4, 1)]


def build_model():
    import torch
    import torch.nn as nn
    import torch.nn.functional as F

    class UNet(nn.Module):
        def __init__(self):
            super().__init__()
            self.convs = nn.ModuleList(nn.Conv2d(ci, co, k, padding=k // 2) for ci, co, k in LAYERS)

        def forward(self, x):  # x [n][8][H][W]
            c = self.convs
            e1 = F.relu(c[1](F.relu(c[0](x))))
            e2 = F.relu(c[3](F.relu(c[2](F.avg_pool2d(e1, 2)))))
            e3 = F.relu(c[5](F.relu(c[4](F.avg_pool2d(e2, 2)))))
            d2 = F.relu(c[7](F.relu(c[6](torch.cat([F.interpolate(e3, scale_factor=2, mode="nearest"), e2], 1)))))
            d1 = F.relu(c[9](F.relu(c[8](torch.cat([F.interpolate(d2, scale_factor=2, mode="nearest"), e1], 1)))))
            return c[10](d1)

    return UNet()


def input_canvas(features, device):
    """[n][8][H][W]: the six features and r/R, z/H at the pixel centres
    (the channel order of the library's k_ws_input)."""
    import torch
    f = torch.as_tensor(np.asarray(features, dtype=np.float32), device=device)
    n = f.shape[0]
    x = torch.empty((n, 8, H, W), device=device)
    x[:, :6] = f[:, :, None, None]
    x[:, 6] = ((torch.arange(W, device=device) + 0.5) / W)[None, None, :]
    x[:, 7] = ((torch.arange(H, device=device) + 0.5) / H)[None, :, None]
    return x


def to_canvas(pb, m, device):
    """Fields of one domain (moments [u_r, u_z, u_theta, T] on its grid) onto
    the canvas: pixel (i_z, i_r) sits at r = (i_r + 1/2)/W r_wall, z =
    z_bottom + (i_z + 1/2)/H height, sampled bilinearly from the nodes."""
    import torch
    import torch.nn.functional as F
    g = I.warm_start_geometry(pb)
    r = (torch.arange(W, device=device) + 0.5) / W * g["r_wall"]
    z = g["z_bottom"] + (torch.arange(H, device=device) + 0.5) / H * g["height"]
    jn = (r - g["r_first"]) / max(pb.nr - 1, 1) * 2 - 1
    kn = (z - g["z_first"]) / max(pb.nz - 1, 1) * 2 - 1
    grid = torch.stack(torch.meshgrid(kn, jn, indexing="ij")[::-1], dim=-1)[None]  # [1][H][W][(x, y)]
    src = torch.as_tensor(m, dtype=torch.float32, device=device)[None]
    out = F.grid_sample(src, grid, mode="bilinear", padding_mode="border", align_corners=True)[0]
    out[:3] /= g["u_scale"]
    out[3] -= pb.t_ref
    return out


def solve_sweep(seed, scale, steps, device):
    probs = I.batch_sweep(seed=seed, scale=scale)
    batch = B.Batch(probs, "fp32")
    batch.step(steps)
    res = batch.residuals(allow_nonfinite=True)
    canv, keep = [], []
    for d, pb in enumerate(probs):
        if pb.temperature:
            m = batch.moments(d, B.UR | B.UZ | B.UTH | B.T, dtype=np.float32)
        else:  # no temperature: T = T_ref
            m3 = batch.moments(d, B.UR | B.UZ | B.UTH, dtype=np.float32)
            m = np.concatenate([m3, np.full((1,) + m3.shape[1:], pb.t_ref, dtype=np.float32)])
        if np.all(np.isfinite(m)):  # a draw that blew up (grid Reynolds number too high) is dropped
            canv.append(to_canvas(pb, m, device))
            keep.append(d)
    batch.close()
    feats = np.array([I.warm_start_features(probs[d]) for d in keep], dtype=np.float32)
    import torch
    return feats, torch.stack(canv), res[keep, 0]


def bf16_bits(t):
    """float32 tensor -> BF16 bit patterns (round to nearest even), numpy uint16."""
    u = t.detach().float().contiguous().cpu().numpy().view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def pack(model):
    parts = []
    for conv in model.convs:
        w = conv.weight  # [Cout][Cin][k][k]
        parts.append(bf16_bits(w.permute(0, 2, 3, 1).reshape(-1)) if w.shape[-1] == 3 else bf16_bits(w.reshape(-1)))
        parts.append(bf16_bits(conv.bias))
    return np.concatenate(parts)


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweeps", type=int, default=7)
    ap.add_argument("--scale", type=float, default=0.5)
    ap.add_argument("--steps", type=int, default=600000)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--out", default=os.path.join(HERE, "warm_start_weights.npz"))
    args = ap.parse_args()
    dev = torch.device("cuda")
    torch.manual_seed(0)
    t0 = time.time()
    feats, canv, res = [], [], []
    for s in range(1, args.sweeps + 1):
        f, c, r = solve_sweep(s, args.scale, args.steps, dev)
        feats.append(f)
        canv.append(c)
        res.append(r)
        print(f"sweep {s}: {time.time() - t0:.0f} s, {len(f)} finite draws, median residual {np.median(r):.2e}",
              flush=True)
    ftr, ctr = np.concatenate(feats[:-1]), torch.cat(canv[:-1])
    fte, cte = feats[-1], canv[-1]
    xtr, xte = input_canvas(ftr, dev), input_canvas(fte, dev)
    model = build_model().to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=1e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, args.iters)
    g = torch.Generator(device="cpu").manual_seed(1)
    for it in range(args.iters):
        idx = torch.randint(0, xtr.shape[0], (args.batch,), generator=g)
        with torch.autocast("cuda", dtype=torch.bfloat16):
            pred = model(xtr[idx])
        loss = torch.mean((pred.float() - ctr[idx]) ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
        sched.step()
        if it % 500 == 0 or it == args.iters - 1:
            with torch.no_grad(), torch.autocast("cuda", dtype=torch.bfloat16):
                test = torch.mean((model(xte).float() - cte) ** 2).item()
            print(f"iter {it}: train {loss.item():.3e} held-out {test:.3e} ({time.time() - t0:.0f} s)", flush=True)
    bits = pack(model)
    assert bits.size == B.lib().axlbm_ws_weight_count()
    np.savez_compressed(args.out, weights=bits,
                        meta=json.dumps(dict(sweeps=args.sweeps, scale=args.scale, steps=args.steps, iters=args.iters,
                                             held_out_mse=test)))
    print(f"wrote {args.out} ({bits.size} weights), {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
