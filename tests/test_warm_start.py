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
    assert B.lib().axlbm_ws_weight_count() == WS.weight_count() == 473092


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
