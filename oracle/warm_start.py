"""CPU reference of the warm-start network and its resampling (test
infrastructure: only tests/ use it; the product path runs the CUDA kernels).

Plain numpy in float64 with the BF16 weights widened exactly: every 3x3
convolution is written as nine shifted matrix products over the zero-padded
input, the pooling and upsampling as array reshapes, so that each layer can
be read against the architecture the library documents (a four-level U-Net
8 -> 32 -> 32 | pool | 32 -> 64 -> 64 | pool | 64 -> 96 -> 96 | pool |
96 -> 128 -> 128 | up, concat | 224 -> 96 -> 96 | up, concat | 160 -> 64 ->
64 | up, concat | 96 -> 32 -> 32 | 1x1 32 -> 4, ReLU after every 3x3
convolution, canvas 256 (z) x 128 (r)).
"""
from __future__ import annotations

import numpy as np

H, W = 256, 128
CHANNELS = (32, 64, 96, 128)  # per level
# encoder levels 0-3 (two 3x3 layers each), decoder levels 2, 1, 0 (two each), the 1x1 head
LAYERS = [(8, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 96, 3), (96, 96, 3), (96, 128, 3),
          (128, 128, 3), (224, 96, 3), (96, 96, 3), (160, 64, 3), (64, 64, 3), (96, 32, 3), (32, 32, 3),
          (32, 4, 1)]


def weight_count() -> int:
    return sum(co * ci * k * k + co for ci, co, k in LAYERS)


def bf16_to_float(bits: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) to float64, exactly."""
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def float_to_bf16(x: np.ndarray) -> np.ndarray:
    """float to BF16 bit patterns, round to nearest even (finite inputs)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def unpack(bits: np.ndarray):
    """[(kernel [Cout][ky][kx][Cin] or [Cout][Cin], bias [Cout]), ...] as float64."""
    v = bf16_to_float(np.asarray(bits).ravel())
    out, off = [], 0
    for ci, co, k in LAYERS:
        n = co * ci * k * k
        w = v[off:off + n].reshape((co, k, k, ci) if k == 3 else (co, ci))
        off += n
        out.append((w, v[off:off + co]))
        off += co
    assert off == v.size
    return out


def conv3(x, w, b):
    """3x3 convolution, zero padding 1, NHWC; w [Cout][ky][kx][Cin]."""
    n, h, wd, _ = x.shape
    xp = np.zeros((n, h + 2, wd + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, w.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + h, kx:kx + wd] @ w[:, ky, kx, :].T
    return y


def relu_bf16(y):
    """ReLU, then rounding to BF16 (the library stores activations in BF16)."""
    return bf16_to_float(float_to_bf16(np.maximum(y, 0.0)))


def pool(x):
    n, h, w, c = x.shape
    return bf16_to_float(float_to_bf16(x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))))


def up_concat(deep, skip):
    return np.concatenate([deep.repeat(2, axis=1).repeat(2, axis=2), skip], axis=3)


def input_canvas(features):
    f = np.asarray(features, dtype=np.float64).reshape(-1, 6)
    n = f.shape[0]
    x = np.zeros((n, H, W, 8))
    x[..., :6] = f[:, None, None, :]
    x[..., 6] = ((np.arange(W) + 0.5) / W)[None, None, :]
    x[..., 7] = ((np.arange(H) + 0.5) / H)[None, :, None]
    return bf16_to_float(float_to_bf16(x))


def forward(bits, features) -> np.ndarray:
    """Canvases [n][4][H][W] of the network with weights `bits` (uint16)."""
    L = unpack(bits)
    x = input_canvas(features)
    levels = len(CHANNELS)
    skips = []
    for lev in range(levels):  # encoder
        if lev:
            x = pool(x)
        x = relu_bf16(conv3(relu_bf16(conv3(x, *L[2 * lev])), *L[2 * lev + 1]))
        skips.append(x)
    for j, lev in enumerate(range(levels - 2, -1, -1)):  # decoder, from the bottom up
        first = 2 * levels + 2 * j
        x = relu_bf16(conv3(relu_bf16(conv3(up_concat(x, skips[lev]), *L[first])), *L[first + 1]))
    wh, bh = L[-1]
    y = x @ wh.T + bh
    return np.transpose(y, (0, 3, 1, 2))


def fields(canvas, geometry, nr, nz, rho0, t_ref):
    """Fields [5][nz][nr] of one domain from its canvas [4][H][W]: bilinear
    at (r / r_wall, (z - z_bottom) / height) with pixel centres at
    ((i + 1/2)/W, (j + 1/2)/H), clamped to the canvas."""
    g = geometry
    r = g["r_first"] + np.arange(nr)
    z = g["z_first"] + np.arange(nz)
    x = np.clip(r / g["r_wall"] * W - 0.5, 0.0, W - 1.0)
    y = np.clip((z - g["z_bottom"]) / g["height"] * H - 0.5, 0.0, H - 1.0)
    x0 = np.minimum(x.astype(int), W - 2)
    y0 = np.minimum(y.astype(int), H - 2)
    fx, fy = (x - x0)[None, :], (y - y0)[:, None]
    out = np.empty((5, nz, nr))
    out[0] = rho0
    for c in range(4):
        p = canvas[c]
        v = ((1 - fy) * ((1 - fx) * p[np.ix_(y0, x0)] + fx * p[np.ix_(y0, x0 + 1)])
             + fy * ((1 - fx) * p[np.ix_(y0 + 1, x0)] + fx * p[np.ix_(y0 + 1, x0 + 1)]))
        out[1 + c] = g["u_scale"] * v if c < 3 else t_ref + v
    return out
