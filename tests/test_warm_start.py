"""The warm-start network (learned initial fields of a batch).

CPU: the numpy reference's pieces against brute force (BF16 rounding, a
3x3 convolution written pixel by pixel, a network whose kernels are zero)
and the weight count against the library.  GPU: the library's forward pass
against the reference on seeded random weights (BF16 activations: agreement
to a few BF16 ulps of the output scale), the resampling onto domain grids,
and a batch started from the network's fields equals one started from the
same fields through axlbm_batch_set_fields_all.
"""
import numpy as np
import pytest

from oracle import warm_start as WS
from paper_1003_0282_gb300 import inputs as I


def random_weights(seed, gain=1.0):
    """He-scaled random kernels and small biases, as BF16 bits."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, k in WS.LAYERS:
        fan_in = ci * k * k
        parts.append(rng.normal(0.0, gain * np.sqrt(2.0 / fan_in), co * fan_in))
        parts.append(rng.uniform(-0.05, 0.05, co))
    return WS.float_to_bf16(np.concatenate(parts))


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3])
    got = WS.bf16_to_float(WS.float_to_bf16(x))
    assert got[0] == 1.0 and got[1] == 1.0  # ties to even
    assert got[2] == 1.0 + 2 ** -7
    assert got[3] == 1.0 + 2 ** -6          # tie rounds up to the even neighbour
    assert got[4] == -2.5
    assert abs(got[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_conv3_against_brute_force():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 4, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = WS.conv3(x, w, b)
    for n in range(2):
        for i in range(5):
            for j in range(4):
                for o in range(2):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            ii, jj = i + ky - 1, j + kx - 1
                            if 0 <= ii < 5 and 0 <= jj < 4:
                                s += w[o, ky, kx] @ x[n, ii, jj]
                    assert abs(y[n, i, j, o] - s) <= 1e-12


def test_zero_kernels_give_the_head_bias():
    bits = np.zeros(WS.weight_count(), dtype=np.uint16)
    bias = WS.float_to_bf16(np.array([0.25, -0.5, 1.0, 2.0]))
    bits[-4:] = bias
    out = WS.forward(bits, np.zeros((1, 6)))
    for c, v in enumerate([0.25, -0.5, 1.0, 2.0]):
        assert np.all(out[0, c] == v)


def test_weight_count_matches_the_library():
    from paper_1003_0282_gb300 import axlbm as B
    assert B.lib().axlbm_ws_weight_count() == WS.weight_count() == 906628


@pytest.fixture(scope="module")
def Bgpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_0282_gb300 import build
    build.build()
    from paper_1003_0282_gb300 import axlbm
    return axlbm


@pytest.mark.gpu
def test_forward_pass_matches_the_reference(Bgpu):
    bits = random_weights(11)
    rng = np.random.default_rng(12)
    feats = rng.uniform(-1, 1, (9, 6))  # two chunks of canvases
    ws = Bgpu.WarmStart(bits)
    got = ws.predict(feats).cpu().numpy()
    ws.close()
    want = WS.forward(bits, feats)
    scale = np.max(np.abs(want))
    err = np.max(np.abs(got - want)) / scale
    assert err <= 3e-2, err
    assert np.sqrt(np.mean((got - want) ** 2)) / scale <= 3e-3


@pytest.mark.gpu
def test_resampling_matches_the_reference(Bgpu):
    import torch
    rng = np.random.default_rng(13)
    probs = [I.rotating_lid_cavity(nr=40, aspect=2.2, re=700.0),
             I.wheeler_cell(nr=33, re_x=300.0, prandtl=5.0, grashof=1e5),
             I.Problem(nr=21, nz=30, tau=0.7, inner="axis_node", outer="nee", z_lo="nee", z_hi="nee", swirl=True,
                       omega={"hi": 0.002})]
    canvas = rng.normal(size=(len(probs), 4, WS.H, WS.W))
    ws = Bgpu.WarmStart(random_weights(1))
    got = ws.fields(torch.tensor(canvas, dtype=torch.float32, device="cuda"), probs).cpu().numpy()
    ws.close()
    off = 0
    for d, pb in enumerate(probs):
        want = WS.fields(canvas[d].astype(np.float32).astype(np.float64), I.warm_start_geometry(pb), pb.nr, pb.nz,
                         pb.rho0, pb.t_ref)
        part = got[off:off + 5 * pb.cells].reshape(5, pb.nz, pb.nr)
        assert np.max(np.abs(part - want)) <= 1e-5 * max(1.0, np.max(np.abs(want))), d
        off += 5 * pb.cells


@pytest.mark.gpu
def test_batch_started_from_the_network(Bgpu):
    probs = I.batch_sweep(scale=0.25)[:12] + I.batch_sweep(scale=0.25)[256:260]
    ws = Bgpu.WarmStart(random_weights(3, gain=0.3))
    a = Bgpu.Batch(probs, "fp32")
    canvas = ws.start(a, probs)
    fields = ws.fields(canvas, probs).cpu().numpy()
    b = Bgpu.Batch(probs, "fp32")
    b.set_fields_all(fields)
    for d in range(len(probs)):
        fa, ga, ha = a.get_populations(d)
        fb, gb, hb = b.get_populations(d)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), d
    a.step(4)
    b.step(4)
    assert np.array_equal(a.residuals(), b.residuals())
    a.close()
    b.close()
    ws.close()


def torch_reference(bits, feats):
    """FP32 PyTorch reference of the network (weights widened from BF16 and
    leaf tensors that take gradients), for the training tests."""
    import torch
    import torch.nn.functional as F
    v = torch.tensor(WS.bf16_to_float(bits), dtype=torch.float32, device="cuda")
    params, off = [], 0
    for ci, co, k in WS.LAYERS:
        n = co * ci * k * k
        w = v[off:off + n].reshape(co, k, k, ci).permute(0, 3, 1, 2).contiguous() if k == 3 else \
            v[off:off + n].reshape(co, ci, 1, 1).contiguous()
        off += n
        b = v[off:off + co].clone()
        off += co
        params += [w.requires_grad_(True), b.requires_grad_(True)]
    f = torch.as_tensor(np.asarray(feats, dtype=np.float32), device="cuda")
    n = f.shape[0]
    x = torch.empty((n, 8, WS.H, WS.W), device="cuda")
    x[:, :6] = f[:, :, None, None]
    x[:, 6] = ((torch.arange(WS.W, device="cuda") + 0.5) / WS.W)[None, None, :]
    x[:, 7] = ((torch.arange(WS.H, device="cuda") + 0.5) / WS.H)[None, :, None]
    x = x.to(torch.bfloat16).float()
    c = lambda i, t: F.conv2d(t, params[2 * i], params[2 * i + 1], padding=1 if WS.LAYERS[i][2] == 3 else 0)
    levels = len(WS.CHANNELS)
    skips = []
    for lev in range(levels):
        if lev:
            x = F.avg_pool2d(x, 2)
        x = F.relu(c(2 * lev + 1, F.relu(c(2 * lev, x))))
        skips.append(x)
    for j, lev in enumerate(range(levels - 2, -1, -1)):
        first = 2 * levels + 2 * j
        x = F.relu(c(first + 1, F.relu(c(first, torch.cat([F.interpolate(x, scale_factor=2, mode="nearest"),
                                                            skips[lev]], 1)))))
    return c(len(WS.LAYERS) - 1, x), params


def packed_grad(params):
    """Gradients of the reference's parameters in the library's weight packing."""
    out = []
    for i, (ci, co, k) in enumerate(WS.LAYERS):
        g = params[2 * i].grad
        out.append((g.permute(0, 2, 3, 1) if k == 3 else g).reshape(-1))
        out.append(params[2 * i + 1].grad.reshape(-1))
    import torch
    return torch.cat(out).cpu().numpy().astype(np.float64)


@pytest.mark.gpu
def test_training_gradient_matches_autograd(Bgpu):
    """The library's backward pass against PyTorch autograd in FP32 (the
    library keeps activations and their gradients in BF16): the loss, and per
    layer the kernel and bias gradients in norm and direction; lr = 0 leaves
    the weights as they were."""
    import torch
    bits = random_weights(21)
    rng = np.random.default_rng(22)
    feats = rng.uniform(-1, 1, (3, 6)).astype(np.float32)
    target = torch.tensor(rng.normal(0.0, 0.1, (3, 4, WS.H, WS.W)), dtype=torch.float32, device="cuda")
    ws = Bgpu.WarmStart(bits)
    loss = ws.train_step(torch.tensor(feats, device="cuda"), target, lr=0.0)
    g = ws.last_gradient().astype(np.float64)
    assert np.array_equal(ws.weights(), bits)
    ws.close()
    out, params = torch_reference(bits, feats)
    ref = torch.mean((out - target) ** 2)
    ref.backward()
    assert abs(loss - ref.item()) <= 2e-2 * ref.item()
    gr = packed_grad(params)
    off = 0
    for ci, co, k in WS.LAYERS:
        for n in (co * ci * k * k, co):
            a, b = g[off:off + n], gr[off:off + n]
            off += n
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            assert rel <= 0.08 and cos >= 0.995, (ci, co, k, n, rel, cos)
    assert off == g.size


@pytest.mark.gpu
def test_training_reduces_the_loss_deterministically(Bgpu):
    """A few Adam steps on a learnable target (each canvas channel a smooth
    function of the features) lower the loss; two runs give the same weights
    bit for bit."""
    import torch
    rng = np.random.default_rng(23)
    feats = torch.tensor(rng.uniform(-1, 1, (8, 6)), dtype=torch.float32, device="cuda")
    r = (torch.arange(WS.W, device="cuda") + 0.5) / WS.W
    z = (torch.arange(WS.H, device="cuda") + 0.5) / WS.H
    target = torch.stack([feats[:, c, None, None] * torch.sin(np.pi * r)[None, None, :] * z[None, :, None]
                          for c in range(4)], dim=1).contiguous()
    runs = []
    for _ in range(2):
        ws = Bgpu.WarmStart(random_weights(24, gain=0.5))
        first = ws.loss(feats, target)
        for _ in range(40):
            ws.train_step(feats, target, lr=3e-3)
        runs.append((first, ws.loss(feats, target), ws.weights()))
        ws.close()
    (l0, l1, w1), (m0, m1, w2) = runs
    assert l0 == m0 and l1 == m1 and np.array_equal(w1, w2)
    assert l1 <= 0.5 * l0, (l0, l1)


@pytest.mark.gpu
def test_canvas_from_fields_matches_numpy(Bgpu):
    """axlbm_ws_to_canvas (the training targets) against a numpy bilinear
    sample of the node values at every pixel centre."""
    import torch
    probs = [I.rotating_lid_cavity(nr=37, aspect=2.0, re=500.0),
             I.wheeler_cell(nr=29, re_x=300.0, prandtl=5.0, grashof=1e5),
             I.Problem(nr=19, nz=27, tau=0.7, inner="axis_node", outer="nee", z_lo="nee", z_hi="nee", swirl=True,
                       omega={"hi": 0.002})]
    rng = np.random.default_rng(25)
    moms = [rng.normal(size=(4, pb.nz, pb.nr)) for pb in probs]
    packed = torch.tensor(np.concatenate([m.ravel() for m in moms]), dtype=torch.float32, device="cuda")
    ws = Bgpu.WarmStart(random_weights(1))
    got = ws.to_canvas(packed, probs).cpu().numpy()
    ws.close()
    for d, pb in enumerate(probs):
        g = I.warm_start_geometry(pb)
        m = moms[d].astype(np.float32).astype(np.float64)
        r = (np.arange(WS.W) + 0.5) / WS.W * g["r_wall"]
        z = g["z_bottom"] + (np.arange(WS.H) + 0.5) / WS.H * g["height"]
        x = np.clip(r - g["r_first"], 0, pb.nr - 1)
        y = np.clip(z - g["z_first"], 0, pb.nz - 1)
        x0 = np.minimum(x.astype(int), pb.nr - 1)
        y0 = np.minimum(y.astype(int), pb.nz - 1)
        x1, y1 = np.minimum(x0 + 1, pb.nr - 1), np.minimum(y0 + 1, pb.nz - 1)
        fx, fy = (x - x0)[None, :], (y - y0)[:, None]
        for c in range(4):
            p = m[c]
            v = ((1 - fy) * ((1 - fx) * p[np.ix_(y0, x0)] + fx * p[np.ix_(y0, x1)])
                 + fy * ((1 - fx) * p[np.ix_(y1, x0)] + fx * p[np.ix_(y1, x1)]))
            want = v / g["u_scale"] if c < 3 else v - pb.t_ref
            assert np.max(np.abs(got[d, c] - want)) <= 1e-5 * max(1.0, np.max(np.abs(want))), (d, c)


def test_training_script_initial_weights():
    """The trainer's starting weights: the library's packing and count, every
    value inside its layer's bound 1/sqrt(fan_in), and the BF16 rounding of
    the trainer equal to the reference's."""
    from paper_1003_0282_gb300 import warm_start_train as T
    assert T.LAYERS == WS.LAYERS
    bits = T.initial_weights(5)
    assert bits.dtype == np.uint16 and bits.size == WS.weight_count()
    off = 0
    v = WS.bf16_to_float(bits)
    for ci, co, k in WS.LAYERS:
        n = co * ci * k * k + co
        bound = 1.0 / np.sqrt(ci * k * k)
        assert np.max(np.abs(v[off:off + n])) <= bound * (1 + 2 ** -7)
        off += n
    x = np.random.default_rng(6).normal(size=1000)
    assert np.array_equal(T.bf16_bits(x), WS.float_to_bf16(x))
